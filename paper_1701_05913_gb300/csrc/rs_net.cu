// Learned pressure stage (placeholder until the network kernels land).
#include "rs_internal.cuh"

int rs_net_apply_pressure(rs_pc *M, const double *rp, double *zp, const int *skip)
{
    (void)M; (void)rp; (void)zp; (void)skip;
    return RS_ERR_INVALID_ARG;
}
