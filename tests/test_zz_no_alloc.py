"""rs_vec_mdot_noalloc: the multi-dot product that allocates no device memory,
for callers that cannot call cudaMalloc (for instance while a stream is being
captured into a graph, or when the host owns all device memory).  Its output
must agree with the ordinary entry point, rs_vec_dot, and with the oracle's
dot, column by column, on two calls in a row (the calls share one static
scratch array).  This file is
collected last so that a run stopping at the first failure has run the rest."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _mdot(rs, V, w, h, k, stream):
    n = w.numel()
    ld = V.shape[1]
    return rs.lib().rs_vec_mdot_noalloc(C.c_void_p(V.data_ptr()), ld, n, k, C.c_void_p(w.data_ptr()),
                                        C.c_void_p(h.data_ptr()), C.c_void_p(stream.cuda_stream))


def test_mdot_noalloc_matches_vec_dot(rs, orc):
    import torch
    ctx = rs.Context(0)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(7)
    for call, (n, k) in enumerate([(1000003, 31), (77777, 64)]):
        ld = n + 5
        V = torch.from_numpy(rng.standard_normal((k, ld))).cuda()
        w = torch.from_numpy(rng.standard_normal(n)).cuda()
        h = torch.full((k,), np.nan, dtype=torch.float64, device="cuda")
        assert _mdot(rs, V, w, h, k, stream) == rs.OK
        torch.cuda.synchronize()
        wv = rs.Vec(ctx, w)
        wh, Vh = w.cpu().numpy(), V.cpu().numpy()
        for j in range(k):
            ref = rs.vec_dot(rs.Vec(ctx, V[j, :n]), wv)
            scale = float((V[j, :n].abs() * w.abs()).sum())
            assert abs(float(h[j]) - ref) <= 1e-13 * scale, (call, j)
            # and the oracle's sequential dot (Fig. 12)
            assert abs(float(h[j]) - orc.dot(Vh[j, :n], wh)) <= 1e-13 * scale, (call, j)


def test_mdot_noalloc_rejects_too_many_columns(rs):
    import torch
    stream = torch.cuda.current_stream()
    V = torch.zeros((65, 10), dtype=torch.float64, device="cuda")
    w = torch.zeros(10, dtype=torch.float64, device="cuda")
    h = torch.zeros(65, dtype=torch.float64, device="cuda")
    assert _mdot(rs, V, w, h, 65, stream) == rs.ERR_INVALID_ARG
    assert _mdot(rs, V, w, h, 0, stream) == rs.ERR_INVALID_ARG
