// Plain FP64 complex product C = alpha * X conj(Y)^T (DFMA, register tiled).
//
// Both commutator products of the IsoMP sweep (Sec. 3.1) have a right factor
// in su(N): Y[k, j] = -conj(Y[j, k]), so X Y = -X conj(Y)^T and both operands
// are read row by row (K contiguous).  This is the reference-precision form of
// the product; on GB300 its bound is the FP64 pipe.
#include "zt_internal.h"

namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
}

__global__ void __launch_bounds__(NT)
zgemm_fp64_kernel(const double2* __restrict__ X, const double2* __restrict__ Y, double2* __restrict__ C,
                  double alpha, int N, int lower_only, const zt_dev_state* st, int gate) {
    if (zt_gate_skip(st, gate)) return;
    const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
    if (lower_only && j0 > i0 + BM - 1) return;   // tile lies strictly above the diagonal
    __shared__ double2 Xs[BK][BM + 1];
    __shared__ double2 Ys[BK][BN + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double cr[4][4], ci[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cr[a][b] = ci[a][b] = 0.0;

    for (int k0 = 0; k0 < N; k0 += BK) {
#pragma unroll
        for (int q = 0; q < (BM * BK) / NT; ++q) {
            const int e = tid + NT * q, row = e >> 4, kk = e & 15;
            const int gk = k0 + kk, gi = i0 + row, gj = j0 + row;
            Xs[kk][row] = (gi < N && gk < N) ? X[(size_t)gi * N + gk] : make_double2(0.0, 0.0);
            Ys[kk][row] = (gj < N && gk < N) ? Y[(size_t)gj * N + gk] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            double2 xa[4], yb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) xa[a] = Xs[kk][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) yb[b] = Ys[kk][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    // x * conj(y) = (xr yr + xi yi) + i (xi yr - xr yi)
                    cr[a][b] = fma(xa[a].x, yb[b].x, cr[a][b]);
                    cr[a][b] = fma(xa[a].y, yb[b].y, cr[a][b]);
                    ci[a][b] = fma(xa[a].y, yb[b].x, ci[a][b]);
                    ci[a][b] = fma(-xa[a].x, yb[b].y, ci[a][b]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = i0 + ty + 16 * a;
        if (i >= N) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = j0 + tx + 16 * b;
            if (j < N) C[(size_t)i * N + j] = make_double2(alpha * cr[a][b], alpha * ci[a][b]);
        }
    }
}

int zt_launch_zgemm_fp64(zt_plan* p, const double2* X, const double2* Y, double2* C, double alpha,
                         int lower_only, cudaStream_t s, int gate) {
    const int N = p->N;
    dim3 grid((N + BN - 1) / BN, (N + BM - 1) / BM);
    // work: FP64 flops over the computed tiles; FP64-equivalent algorithmic flops
    double tiles = (double)grid.x * grid.y;
    if (lower_only) tiles = 0.5 * grid.y * (grid.y + 1.0);
    const double work = tiles * BM * BN * 8.0 * (double)N;
    const double alg = lower_only ? 4.0 * N * (double)N * (N + 1.0) : 8.0 * (double)N * N * N;
    const int t = zt_timer_begin(p, ZT_KERNEL_PRODUCT, work, alg, s);
    zgemm_fp64_kernel<<<grid, NT, 0, s>>>(X, Y, C, alpha, N, lower_only, p->state, gate);
    zt_timer_end(p, t, s);
    p->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "zgemm_fp64_kernel");
    return ZT_OK;
}
