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

__device__ __forceinline__ void zgemm_fp64_body(const double2* __restrict__ X, const double2* __restrict__ Y,
                                                double2* __restrict__ C, double alpha, int N, int lower_only,
                                                const zt_dev_state* st, int gate, int bx, int by) {
    if (zt_gate_skip(st, gate)) return;
    const int i0 = by * BM, j0 = bx * BN;
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

__global__ void __launch_bounds__(NT)
zgemm_fp64_kernel(const double2* __restrict__ X, const double2* __restrict__ Y, double2* __restrict__ C,
                  double alpha, int N, int lower_only, const zt_dev_state* st, int gate) {
    zgemm_fp64_body(X, Y, C, alpha, N, lower_only, st, gate, blockIdx.x, blockIdx.y);
}

// Grouped: each instance's tile grid is flattened (gx tiles per row of tiles).
__global__ void __launch_bounds__(NT) zgemm_fp64_grouped(const Fp64GemmArgs* tab, const int* offs, int n, int gate) {
    const int inst = zt_group_find(offs, n, blockIdx.x);
    const Fp64GemmArgs a = tab[inst];
    const int b = blockIdx.x - offs[inst];
    zgemm_fp64_body(a.X, a.Y, a.C, a.alpha, a.N, a.lower_only, a.st, gate, b % a.gx, b / a.gx);
}

int zt_fp64_gemm_args(zt_plan* p, const double2* X, const double2* Y, double2* C, double alpha, int lower_only,
                      Fp64GemmArgs* out, int* ctas) {
    const int N = p->N;
    out->X = X;
    out->Y = Y;
    out->C = C;
    out->alpha = alpha;
    out->N = N;
    out->lower_only = lower_only;
    out->gx = (N + BN - 1) / BN;
    out->st = p->state;
    out->gate = ZT_GATE_NONE;
    *ctas = out->gx * ((N + BM - 1) / BM);
    return ZT_OK;
}

int zt_fp64_gemm_grouped(const Fp64GemmArgs* tab, const int* offs, int n, int total, cudaStream_t s, int gate) {
    zgemm_fp64_grouped<<<total, NT, 0, s>>>(tab, offs, n, gate);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "zgemm_fp64_grouped");
    return ZT_OK;
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
