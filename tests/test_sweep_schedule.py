"""The schedule of the sync-free triangular sweeps, on the host (no GPU):
segments, levels and runs from rs_sweep_schedule, checked against the
pattern they come from.

A warp takes a run of segments on one ticket and, after the first segment,
finds every later one by fixed strides; it may wait only for rows held by
runs with earlier tickets, or by earlier segments of its own run.  These
tests check those properties on grid patterns (where runs form), on grids
with entries knocked out at random (where runs break and restart), and on
random patterns (where they do not form), for both sweeps.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth


@pytest.fixture(scope="module")
def rs():
    """The binding, built here; these calls make no device call."""
    import paper_1701_05913_gb300 as rs_mod
    rs_mod.build()
    return rs_mod


def _pattern_7pt(shape, drop=0.0, seed=0):
    d = synth.pressure_7pt(synth.Grid(*shape), 1)
    A = sp.csr_matrix((np.ones(d["col"].size), d["col"], d["rowptr"]), shape=(d["n"], d["n"]))
    if drop:
        C = A.tocoo()
        rng = np.random.default_rng(seed)
        keep = (C.row == C.col) | (rng.random(C.nnz) >= drop)
        A = sp.csr_matrix((C.data[keep], (C.row[keep], C.col[keep])), shape=A.shape)
    A.sort_indices()
    return A


def _pattern_random(n, density, seed):
    R = sp.random(n, n, density=density, random_state=seed, format="csr")
    A = (R + sp.eye(n)).tocsr()
    A.data[:] = 1.0
    A.sort_indices()
    return A


def _check(rs, A, lower, run_cap=1 << 30):
    n = A.shape[0]
    ptr, col = A.indptr, A.indices
    S = rs.sweep_schedule(ptr, col, lower=lower, run_cap=run_cap)
    row0, lev, runs = S["row0"], S["level"], S["runs"]
    nseg = row0.size - 1
    # segments: consecutive, at most 32 rows, covering [0, n)
    assert row0[0] == 0 and row0[-1] == n
    assert (np.diff(row0) >= 1).all() and (np.diff(row0) <= 32).all()
    seg_of = np.repeat(np.arange(nseg), np.diff(row0))

    def reads(i):   # the rows row i reads in this sweep
        c = col[ptr[i]:ptr[i + 1]]
        return c[c < i] if lower else c[c > i]

    # levels: one more than the highest level among the segments read
    order = range(nseg) if lower else range(nseg - 1, -1, -1)
    want = np.zeros(nseg, int)
    for s in order:
        l = 0
        for i in range(row0[s], row0[s + 1]):
            for c in reads(i):
                if not (row0[s] <= c < row0[s + 1]):
                    l = max(l, want[seg_of[c]] + 1)
        want[s] = l
    assert np.array_equal(lev, want)
    assert S["nlevels"] == want.max() + 1
    # runs: a partition of the segments, each segment k found by the strides
    run_of, pos = np.full(nseg, -1), np.full(nseg, -1)
    for R, (s0, cnt, dseg, drow, dent) in enumerate(runs):
        assert 1 <= cnt <= run_cap
        for k in range(cnt):
            s = s0 + k * dseg
            assert run_of[s] == -1
            run_of[s], pos[s] = R, k
            assert row0[s] == row0[s0] + k * drow
            assert row0[s + 1] - row0[s] == row0[s0 + 1] - row0[s0]
            if k >= 2:   # from the second segment on, the columns shift with the rows
                p = s - dseg
                for t in range(row0[s + 1] - row0[s]):
                    assert np.array_equal(reads(row0[s] + t), reads(row0[p] + t) + drow)
            if k >= 1:   # later segments: the only in-segment reads are the adjacent row
                for i in range(row0[s], row0[s + 1]):
                    inside = [c for c in reads(i) if row0[s] <= c < row0[s + 1]]
                    assert inside in ([], [i - 1] if lower else [i + 1])
                    assert len(reads(i)) <= 4
    assert (run_of >= 0).all()
    # deadlock-freedom: every row read lies in an earlier run, or earlier in
    # the same run (held by a warp that took an earlier ticket or by itself)
    for s in range(nseg):
        for i in range(row0[s], row0[s + 1]):
            for c in reads(i):
                q = seg_of[c]
                if q == s:
                    continue
                assert run_of[q] < run_of[s] or (run_of[q] == run_of[s] and pos[q] < pos[s]), (s, q)
    # tickets go in the level order of the runs' first segments
    first_lev = lev[runs[:, 0]]
    assert (np.diff(first_lev) >= 0).all()
    return S


@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("shape", [(64, 16, 8), (40, 12, 6), (7, 5, 3), (50, 40, 1), (96, 3, 20)])
def test_grid_runs_follow_the_y_lines(rs, shape, lower):
    nx, ny, nz = shape
    S = _check(rs, _pattern_7pt(shape), lower)
    xsegs = -(-nx // 32)
    assert len(S["runs"]) == xsegs * nz
    assert (S["runs"][:, 1] == ny).all()
    assert S["nlevels"] == xsegs + ny + nz - 2


@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("drop,seed", [(0.002, 1), (0.01, 2), (0.05, 3)])
def test_grids_with_entries_knocked_out(rs, lower, drop, seed):
    """Missing entries break the strides: runs end and new ones start, and
    the schedule stays deadlock-free."""
    S = _check(rs, _pattern_7pt((48, 20, 10), drop, seed), lower)
    assert len(S["runs"]) >= 2 * 10


@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("cap", [1, 2, 5])
def test_capped_runs(rs, lower, cap):
    S = _check(rs, _pattern_7pt((40, 12, 6)), lower, run_cap=cap)
    if cap == 1:
        assert (S["runs"][:, 1] == 1).all() and len(S["runs"]) == S["row0"].size - 1
    else:
        assert S["runs"][:, 1].max() == cap


@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("n,density,seed", [(300, 0.01, 4), (500, 0.004, 5), (200, 0.05, 6)])
def test_random_patterns_take_one_segment_per_run(rs, lower, n, density, seed):
    S = _check(rs, _pattern_random(n, density, seed), lower)
    assert len(S["runs"]) == S["row0"].size - 1


def test_bad_patterns_rejected(rs):
    A = _pattern_7pt((8, 4, 2))
    C = A.tocoo()
    keep = ~((C.row == 5) & (C.col == 5))            # row 5 without its diagonal
    B = sp.csr_matrix((C.data[keep], (C.row[keep], C.col[keep])), shape=A.shape)
    B.sort_indices()
    for p, c in ((B.indptr, B.indices), (A.indptr, A.indices[::-1].copy())):
        with pytest.raises(rs.RsError) as e:
            rs.sweep_schedule(p, c)
        assert e.value.status == rs.ERR_BAD_PATTERN


def test_malformed_row_pointers_rejected(rs):
    """A decreasing row pointer array, or a negative last entry, is rejected
    before any column index is read (no read past the column array)."""
    for p, c in (([0, 5, 2], [0, 1]), ([0, 1, -3], [0]), ([0, 2, 1, 3], [0, 1, 2])):
        with pytest.raises(rs.RsError) as e:
            rs.sweep_schedule(np.array(p, np.int32), np.array(c, np.int32))
        assert e.value.status == rs.ERR_BAD_PATTERN
