// Split-precision complex product on tcgen05 (placeholder until the kernel lands).
#include "zt_internal.h"

int zt_split_create(zt_plan* p) {
    (void)p;
    return zt_fail(ZT_EINVAL, "ZT_PRECISION_SPLIT is not available in this build");
}

void zt_split_destroy(zt_plan* p) { (void)p; }

int zt_launch_zgemm_split(zt_plan* p, const double2* X, const double2* Y, double2* C, double alpha,
                          int lower_only, cudaStream_t s, int gate) {
    (void)p; (void)X; (void)Y; (void)C; (void)alpha; (void)lower_only; (void)s; (void)gate;
    return zt_fail(ZT_EINVAL, "ZT_PRECISION_SPLIT is not available in this build");
}
