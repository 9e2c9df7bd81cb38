// Stream solve P = Delta_N^{-1} W (Sec. 3.3, Eq. sub_tria_W), segmented.
//
// Diagonal m (0 <= m < N) of the lower triangle holds the N-m unknowns of the
// tridiagonal system T_m x = -w (T_m = -Delta^m, Eq. delta_tria), solved with
// the plan's LDL^T factors:
//     forward   z_i = w_i - l_i z_{i-1}                 (l_0 = 0)
//     backward  x_i = nd_i z_i - l_{i+1} x_{i+1}         (nd_i = -1/d_i)
// Both recurrences are linear, so a segment [kL, kL+L) can be run from a zero
// inflow and corrected afterwards:
//     z_i = z0_i + G_i z_{kL-1},   G_i = prod_{j=kL..i} (-l_j)
//     x_i = x0_i + H_i x_{kL+L},   H_i = prod_{j=i+1..kL+L} (-l_j)
// Three launches, each over tiles of SD diagonals x SL positions:
//   F1  local forward sweep; z0 parked in the lower triangle of P, segment
//       end values (z0, G) to a small array;
//   B1  inflow z_{kL-1} folded from the earlier segments' end values, z fixed
//       up, local backward sweep; x0 parked in P, segment start values (x0, H);
//   B3  inflow x_{kL+L} folded from the later segments' start values, x fixed
//       up, written to the lower triangle and, as -conj, to the upper one.
// The band's elements in rows [r0, r0 + SL + SD) are SD-long contiguous runs
// of each row, so every tile is staged through shared memory with coalesced
// loads and stores.  The singular m = 0 block has its right-hand side mean
// removed before F1 and the mean of its solution removed in B3 (l = 0 mode),
// from per-segment sums of x0 and H.
#include "zt_internal.h"

namespace {
constexpr int SD = 16;             // diagonals per tile
constexpr int SL = 64;             // positions per segment
constexpr int SROWS = SL + SD;     // staged rows per tile
constexpr int STH = 64;            // threads per CTA: 2 per diagonal (re, im) compute, all stage
constexpr size_t TILE_SMEM = (size_t)SROWS * SD * (sizeof(double2) + 2 * sizeof(double));

enum Phase { F1 = 0, B1 = 1, B3 = 2 };


__device__ __forceinline__ void cp16(void* smem, const void* g, bool ok) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(g), "r"(ok ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp8(void* smem, const void* g, bool ok) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(g), "r"(ok ? 8 : 0) : "memory");
}

// (band, segment) of a linear tile index: band b owns ceil((N - b SD) / SL) segments.
__device__ void tile_of(int t, int N, int* band, int* seg) {
    int b = 0;
    for (;;) {
        const int nseg = (N - b * SD + SL - 1) / SL;
        if (t < nseg) break;
        t -= nseg;
        ++b;
    }
    *band = b;
    *seg = t;
}

__device__ double sum_block(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = STH / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}
}  // namespace

template <int PH>
__device__ __forceinline__ void solve_tile_body(const SolveArgs& a, int bid) {
    if (zt_gate_skip(a.st, a.gate)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    double2* tv = reinterpret_cast<double2*>(smem);     // [SROWS][SD] values
    double* tl = reinterpret_cast<double*>(tv + SROWS * SD);   // [SROWS][SD] l
    double* tn = tl + SROWS * SD;                        // [SROWS][SD] nd
    __shared__ double red[STH];
    const int N = a.N, K = a.K;
    int band, k;
    tile_of(bid, N, &band, &k);
    const int m0 = band * SD, r0 = k * SL + m0;
    const int tid = threadIdx.x;

    // ---- stage rows [r0, r0 + SROWS) of the band ----
    const double2* src = (PH == F1) ? a.W : a.P;
    for (int e = tid; e < SROWS * SD; e += STH) {
        const int rr = e / SD, j = e % SD;
        const int r = r0 + rr, c = r - m0 - SD + 1 + j, tt = SD - 1 - j, m = m0 + tt;
        const bool ok = (r < N) && (m < N) && (c >= 0);
        const size_t q = ok ? zt_tri(r, c) : 0;
        cp16(&tv[rr * SD + tt], src + (ok ? (size_t)r * N + c : 0), ok);
        cp8(&tl[rr * SD + tt], a.fl + q, ok);
        if (PH == B1) cp8(&tn[rr * SD + tt], a.fnd + q, ok);
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");

    double mu = 0.0;   // m = 0: mean of the right-hand side (F1) or of x (B3), one part
    const int t = tid >> 1, part = tid & 1;   // diagonal of the tile, re (0) / im (1)
    const bool worker = t < SD;                // threads beyond 2*SD only stage
    const int m = m0 + t;
    const int n = N - m;                       // length of diagonal m (<= 0: none)
    const int i0 = k * SL, i1 = min(i0 + SL, n);   // positions of this segment
    if (PH == F1 && band == 0) {
        double s = 0.0;
        for (int i = tid >> 1; i < N; i += STH / 2) s += reinterpret_cast<const double*>(a.W)[2 * ((size_t)i * N + i) + part];
        // both parts reduce separately: sum over threads of the same parity
        red[tid] = s;
        __syncthreads();
        for (int w = STH / 2; w > 1; w >>= 1) {
            if (tid < w) red[tid] += red[tid + w];
            __syncthreads();
        }
        mu = red[part] / N;
        __syncthreads();
    }
    __syncthreads();

    double* tvd = reinterpret_cast<double*>(tv);
    auto V = [&](int i) -> double& { return tvd[2 * ((i - k * SL + t) * SD + t) + part]; };
    auto Lf = [&](int i) -> double { return tl[(i - k * SL + t) * SD + t]; };
    auto ND = [&](int i) -> double { return tn[(i - k * SL + t) * SD + t]; };
    const size_t sidx = (size_t)m * K + k;

    if (PH == F1) {
        if (worker && m < N && i0 < n) {
            double z = 0.0, G = 1.0;
            for (int i = i0; i < i1; ++i) {
                double w = V(i);
                if (m == 0) w -= mu;
                const double l = Lf(i);
                z = fma(-l, z, w);
                G *= -l;
                V(i) = z;
            }
            reinterpret_cast<double*>(a.seg_z + sidx)[part] = z;
            if (part == 0) a.seg_g[sidx] = G;
        }
    } else if (PH == B1) {
        double xsum = 0.0, hsum = 0.0;
        if (worker && m < N && i0 < n) {
            double c = 0.0;   // z at position i0 - 1
            for (int kk = 0; kk < k; ++kk) {
                const size_t q = (size_t)m * K + kk;
                c = fma(a.seg_g[q], c, reinterpret_cast<const double*>(a.seg_z + q)[part]);
            }
            double G = 1.0;
            for (int i = i0; i < i1; ++i) {   // z = z0 + G c
                G *= -Lf(i);
                V(i) = fma(G, c, V(i));
            }
            double x = 0.0, H;
            H = (i1 < n) ? -Lf(i1) : 0.0;      // couples x_{i1-1} to x_{i1}
            for (int i = i1 - 1; i >= i0; --i) {
                const double lnext = (i + 1 < n) ? Lf(i + 1) : 0.0;
                x = fma(-lnext, x, ND(i) * V(i));
                if (i < i1 - 1) H *= -lnext;
                V(i) = x;
                xsum += x;
                hsum += H;
            }
            reinterpret_cast<double*>(a.seg_x + sidx)[part] = x;
            if (part == 0) a.seg_h[sidx] = H;
            if (m == 0) {
                reinterpret_cast<double*>(a.sum_x + k)[part] = xsum;
                if (part == 0) a.sum_h[k] = hsum;
            }
        }
    } else {   // B3
        if (worker && m < N && i0 < n) {
            const int Km = (n + SL - 1) / SL;
            double d = 0.0;   // x at position i1 (first position of the next segment)
            for (int kk = Km - 1; kk > k; --kk) {
                const size_t q = (size_t)m * K + kk;
                d = fma(a.seg_h[q], d, reinterpret_cast<const double*>(a.seg_x + q)[part]);
            }
            if (m == 0) {   // mean of the whole m = 0 solution from the segment sums
                double tot = 0.0, dd = 0.0;
                for (int kk = Km - 1; kk >= 0; --kk) {
                    const size_t q = (size_t)kk;
                    tot += fma(a.sum_h[q], dd, reinterpret_cast<const double*>(a.sum_x + q)[part]);
                    dd = fma(a.seg_h[q], dd, reinterpret_cast<const double*>(a.seg_x + q)[part]);
                }
                mu = tot / N;
            }
            double H = (i1 < n) ? -Lf(i1) : 0.0;
            for (int i = i1 - 1; i >= i0; --i) {
                if (i < i1 - 1) H *= -Lf(i + 1);
                V(i) = fma(H, d, V(i)) - mu;
            }
        }
    }
    __syncthreads();

    // ---- write back this segment's positions of the lower triangle ----
    for (int e = tid; e < SROWS * SD; e += STH) {
        const int rr = e / SD, j = e % SD;
        const int r = r0 + rr, c = r - m0 - SD + 1 + j, tt = SD - 1 - j, mm = m0 + tt;
        const int i = c;   // position along diagonal mm
        const bool ok = (r < N) && (mm < N) && (c >= 0) && (i >= k * SL) && (i < k * SL + SL);
        if (ok) a.P[(size_t)r * N + c] = tv[rr * SD + tt];
    }
    if (PH == B3) {   // upper triangle: P[i, i+m] = -conj(P[i+m, i]), rows of SD contiguous entries
        for (int e = tid; e < SL * SD; e += STH) {
            const int ii = e / SD, tt = e % SD;
            const int i = k * SL + ii, mm = m0 + tt;
            if (mm == 0 || mm >= N || i >= N - mm) continue;
            const double2 v = tv[(ii + tt) * SD + tt];
            a.P[(size_t)i * N + i + mm] = make_double2(-v.x, v.y);
        }
    }
}

template <int PH>
__global__ void __launch_bounds__(STH) solve_tile_kernel(const SolveArgs a) {
    solve_tile_body<PH>(a, blockIdx.x);
}

// Grouped: one grid over several instances (tile counts prefix-summed in offs).
template <int PH>
__global__ void __launch_bounds__(STH) solve_tile_grouped(const SolveArgs* tab, const int* offs, int n, int gate) {
    const int inst = zt_group_find(offs, n, blockIdx.x);
    SolveArgs a = tab[inst];
    a.gate = gate;
    solve_tile_body<PH>(a, blockIdx.x - offs[inst]);
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
static int solve_tiles(int N) {
    int tiles = 0;
    for (int b = 0; b * SD < N; ++b) tiles += (N - b * SD + SL - 1) / SL;
    return tiles;
}

int zt_solve_create(zt_plan* p) {
    const int N = p->N;
    p->nseg = (N + SL - 1) / SL;
    const size_t ns = (size_t)N * p->nseg;
    ZT_CU(ZT_DMALLOC(p->seg_z, ns * sizeof(double2), p->mstream));
    ZT_CU(ZT_DMALLOC(p->seg_g, ns * sizeof(double), p->mstream));
    ZT_CU(ZT_DMALLOC(p->seg_x, ns * sizeof(double2), p->mstream));
    ZT_CU(ZT_DMALLOC(p->seg_h, ns * sizeof(double), p->mstream));
    ZT_CU(ZT_DMALLOC(p->sum_x, (size_t)p->nseg * sizeof(double2), p->mstream));
    ZT_CU(ZT_DMALLOC(p->sum_h, (size_t)p->nseg * sizeof(double), p->mstream));
    if (!zt_attr_needed(ZT_ATTR_SOLVE)) return ZT_OK;
    ZT_CU(cudaFuncSetAttribute(solve_tile_kernel<F1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM));
    ZT_CU(cudaFuncSetAttribute(solve_tile_kernel<B1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM));
    ZT_CU(cudaFuncSetAttribute(solve_tile_kernel<B3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM));
    ZT_CU(cudaFuncSetAttribute(solve_tile_grouped<F1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM));
    ZT_CU(cudaFuncSetAttribute(solve_tile_grouped<B1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM));
    ZT_CU(cudaFuncSetAttribute(solve_tile_grouped<B3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM));
    return ZT_OK;
}

void zt_solve_destroy(zt_plan* p) {
    zt_dfree(p->seg_z, p->mstream);
    zt_dfree(p->seg_g, p->mstream);
    zt_dfree(p->seg_x, p->mstream);
    zt_dfree(p->seg_h, p->mstream);
    zt_dfree(p->sum_x, p->mstream);
    zt_dfree(p->sum_h, p->mstream);
}

int zt_solve_ctas(int N) { return solve_tiles(N); }

int zt_solve_args(zt_plan* p, const double2* W, double2* P, SolveArgs* out) {
    SolveArgs& a = *out;
    a.W = W;
    a.P = P;
    a.fl = p->fac_l;
    a.fnd = p->fac_nd;
    a.seg_z = p->seg_z;
    a.seg_g = p->seg_g;
    a.seg_x = p->seg_x;
    a.seg_h = p->seg_h;
    a.sum_x = p->sum_x;
    a.sum_h = p->sum_h;
    a.N = p->N;
    a.K = p->nseg;
    a.st = p->state;
    a.gate = ZT_GATE_NONE;
    return ZT_OK;
}

int zt_solve_grouped(const SolveArgs* tab, const int* offs, int n, int total, cudaStream_t s, int gate) {
    solve_tile_grouped<F1><<<total, STH, TILE_SMEM, s>>>(tab, offs, n, gate);
    solve_tile_grouped<B1><<<total, STH, TILE_SMEM, s>>>(tab, offs, n, gate);
    solve_tile_grouped<B3><<<total, STH, TILE_SMEM, s>>>(tab, offs, n, gate);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "solve_tile_grouped");
    return ZT_OK;
}

int zt_launch_stream_solve(zt_plan* p, const double2* W, double2* P, cudaStream_t s, int gate) {
    const int N = p->N;
    SolveArgs a;
    a.W = W;
    a.P = P;
    a.fl = p->fac_l;
    a.fnd = p->fac_nd;
    a.seg_z = p->seg_z;
    a.seg_g = p->seg_g;
    a.seg_x = p->seg_x;
    a.seg_h = p->seg_h;
    a.sum_x = p->sum_x;
    a.sum_h = p->sum_h;
    a.N = N;
    a.K = p->nseg;
    a.st = p->state;
    a.gate = gate;
    const int tiles = solve_tiles(N);
    const double bytes = 8.0 * N * (N + 1.0) + 16.0 * N * N;
    const int t = zt_timer_begin(p, ZT_KERNEL_SOLVE, bytes, bytes, s);
    solve_tile_kernel<F1><<<tiles, STH, TILE_SMEM, s>>>(a);
    solve_tile_kernel<B1><<<tiles, STH, TILE_SMEM, s>>>(a);
    solve_tile_kernel<B3><<<tiles, STH, TILE_SMEM, s>>>(a);
    zt_timer_end(p, t, s);
    p->launches += 3;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "solve_tile_kernel");
    return ZT_OK;
}
