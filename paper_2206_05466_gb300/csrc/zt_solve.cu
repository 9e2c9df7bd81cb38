// Stream solve P = Delta_N^{-1} W (Sec. 3.3, Eq. 14), segmented.
//
// Diagonal m (0 <= m < N) of the lower triangle holds the N-m unknowns of the
// tridiagonal system T_m x = -w (T_m = -Delta^m, Eq. 13), solved with
// the plan's LDL^T factors:
//     forward   z_i = w_i - l_i z_{i-1}                 (l_0 = 0)
//     backward  x_i = nd_i z_i - l_{i+1} x_{i+1}         (nd_i = -1/d_i)
// Both recurrences are linear, so a segment [kL, kL+L) can be run from a zero
// inflow and corrected afterwards:
//     z_i = z0_i + G_i z_{kL-1},   G_i = prod_{j=kL..i} (-l_j)
//     x_i = x0_i + H_i x_{kL+L},   H_i = prod_{j=i+1..kL+L} (-l_j)
// G and H depend only on the factors: the plan computes them once, with their
// segment end/start values and (m = 0) segment sums of H.  Five launches:
//   F1  tiles of SD diagonals x SL positions: local forward sweep, z0 parked
//       in the lower triangle of P, segment end values z0 to a small array;
//   SF  one thread per (diagonal, re/im): the inflow z_{kL-1} of every
//       segment, by the recurrence over the segment end values;
//   B1  tiles: z = z0 + G z_{kL-1} folded into the local backward sweep, x0
//       parked in P, segment start values x0;
//   SB  one thread per (diagonal, re/im): the inflow x_{kL+L} of every
//       segment, and for m = 0 the mean of the whole solution;
//   B3  tiles: x = x0 + H x_{kL+L}, written to the lower triangle and, as
//       -conj, to the upper one.
// The band's elements in rows [r0, r0 + SL + SD) are SD-long contiguous runs
// of each row, so every tile stages them through shared memory with
// coalesced loads and stores.  The factors and products are stored
// diagonal-major (each diagonal padded to 8 entries), so a thread walking its
// diagonal reads them straight from global memory, 8 positions at a time,
// while the dependent FP64 chain runs on registers.  The singular m = 0 block
// has its right-hand side mean removed in F1 and the mean of its solution
// removed in B3 (l = 0 mode).
#include <thread>
#include <vector>

#include "zt_internal.h"

namespace {
constexpr int SD = 16;             // diagonals per tile
constexpr int SL = 32;             // positions per segment (32 measured best: more tiles in flight, short carries)
constexpr int SROWS = SL + SD;     // staged rows per tile
constexpr int STH = 64;            // threads per CTA: 2 per diagonal (re, im) compute, all stage
constexpr int CH = 8;              // positions per register chunk
constexpr size_t TILE_SMEM = (size_t)SROWS * SD * sizeof(double2);
constexpr int SCAN_TH = 128;

enum Phase { F1 = 0, B1 = 1, B3 = 2 };

__device__ __forceinline__ void cp16(void* smem, const void* g, bool ok) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(g), "r"(ok ? 16 : 0) : "memory");
}

// 8 consecutive doubles from a 16-byte aligned address (read-only data)
__device__ __forceinline__ void load8(double (&v)[CH], const double* p) {
#pragma unroll
    for (int u = 0; u < CH; u += 2) {
        const double2 t = __ldg(reinterpret_cast<const double2*>(p + u));
        v[u] = t.x;
        v[u + 1] = t.y;
    }
}

__device__ __forceinline__ double part_of(const double2& v, int part) { return part ? v.y : v.x; }

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
}  // namespace

template <int PH>
__device__ __forceinline__ void solve_tile_body(const SolveArgs& a, int bid) {
    if (zt_gate_skip(a.st, a.gate)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    double2* tv = reinterpret_cast<double2*>(smem);   // [SROWS][SD] values
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
        cp16(&tv[rr * SD + tt], src + (ok ? (size_t)r * N + c : 0), ok);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");

    double mu = 0.0;   // F1, m = 0: mean of the right-hand side, one part
    const int t = tid >> 1, part = tid & 1;   // diagonal of the tile, re (0) / im (1)
    if (PH == F1 && band == 0) {   // overlaps the staging copies
        const double* wd = reinterpret_cast<const double*>(a.W);
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        const int step = STH / 2;
        int i = tid >> 1;
        for (; i + 3 * step < N; i += 4 * step) {
            s0 += wd[2 * ((size_t)i * N + i) + part];
            s1 += wd[2 * ((size_t)(i + step) * N + i + step) + part];
            s2 += wd[2 * ((size_t)(i + 2 * step) * N + i + 2 * step) + part];
            s3 += wd[2 * ((size_t)(i + 3 * step) * N + i + 3 * step) + part];
        }
        for (; i < N; i += step) s0 += wd[2 * ((size_t)i * N + i) + part];
        red[tid] = (s0 + s1) + (s2 + s3);
        __syncthreads();
        for (int w = STH / 2; w > 1; w >>= 1) {   // threads of the same parity reduce together
            if (tid < w) red[tid] += red[tid + w];
            __syncthreads();
        }
        mu = red[part] / N;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();

    const int m = m0 + t;
    const int n = N - m;                           // length of diagonal m (<= 0: none)
    const int i0 = k * SL, i1 = min(i0 + SL, n);   // positions of this segment
    double* tvd = reinterpret_cast<double*>(tv);
    auto V = [&](int i) -> double& { return tvd[2 * ((i - i0 + t) * SD + t) + part]; };

    if (t < SD && m < N && i0 < n) {
        const size_t base = a.dof[m];
        const size_t sidx = (size_t)m * K + k;
        if (PH == F1) {
            const double* L = a.fl + base;
            double z = 0.0;
            for (int j = i0; j < i1; j += CH) {
                double lc[CH], w[CH];
                load8(lc, L + j);
#pragma unroll
                for (int u = 0; u < CH; ++u) w[u] = (j + u < i1) ? V(j + u) : 0.0;
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    if (j + u < i1) {
                        z = fma(-lc[u], z, (m == 0) ? w[u] - mu : w[u]);
                        w[u] = z;
                    }
                }
#pragma unroll
                for (int u = 0; u < CH; ++u)
                    if (j + u < i1) V(j + u) = w[u];
            }
            reinterpret_cast<double*>(a.seg_z + sidx)[part] = z;
        } else if (PH == B1) {
            const double *L = a.fl + base, *ND = a.fnd + base, *G = a.fg + base;
            const double c = part_of(a.cf[sidx], part);   // z at position i0 - 1
            double x = 0.0, xsum = 0.0;
            double lnext = (i1 < n) ? L[i1] : 0.0;        // l at the position after the one in hand
            for (int j = i0 + ((i1 - 1 - i0) / CH) * CH; j >= i0; j -= CH) {
                double lc[CH], nc[CH], gc[CH], v[CH];
                load8(lc, L + j);
                load8(nc, ND + j);
                load8(gc, G + j);
#pragma unroll
                for (int u = 0; u < CH; ++u) v[u] = (j + u < i1) ? V(j + u) : 0.0;
#pragma unroll
                for (int u = CH - 1; u >= 0; --u) {
                    if (j + u < i1) {
                        const double z = fma(gc[u], c, v[u]);   // z = z0 + G c
                        x = fma(-lnext, x, nc[u] * z);
                        v[u] = x;
                        if (m == 0) xsum += x;
                    }
                    lnext = lc[u];   // padding past the diagonal's end holds zeros
                }
#pragma unroll
                for (int u = 0; u < CH; ++u)
                    if (j + u < i1) V(j + u) = v[u];
            }
            reinterpret_cast<double*>(a.seg_x + sidx)[part] = x;
            if (m == 0) reinterpret_cast<double*>(a.sum_x + k)[part] = xsum;
        } else {   // B3
            const double* H = a.fh + base;
            const double d = part_of(a.cb[sidx], part);   // x at position i1
            const double mm = (m == 0) ? part_of(*a.mu, part) : 0.0;
            for (int j = i0; j < i1; j += CH) {
                double hc[CH];
                load8(hc, H + j);
#pragma unroll
                for (int u = 0; u < CH; ++u)
                    if (j + u < i1) V(j + u) = fma(hc[u], d, V(j + u)) - mm;
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

// Inflows of every segment of diagonal m, one part (re/im) per thread.
//   forward:  c_0 = 0, c_{k+1} = G_end(k) c_k + z0_end(k)
//   backward: d_{K-1} = 0, d_{k-1} = H_start(k) d_k + x0_start(k); for m = 0
//             also the mean of the solution, sum_k (sum H(k) d_k + sum x0(k)) / N.
template <bool FWD>
__device__ __forceinline__ void scan_body(const SolveArgs& a, int gid) {
    if (zt_gate_skip(a.st, a.gate)) return;
    const int m = gid >> 1, part = gid & 1;
    if (m >= a.N) return;
    const int n = a.N - m, Km = (n + SL - 1) / SL, K = a.K;
    const size_t row = (size_t)m * K;
    if (FWD) {
        double c = 0.0;
        for (int k0 = 0; k0 < Km; k0 += CH) {
            double zz[CH], gg[CH];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const bool in = k0 + u < Km;
                zz[u] = in ? part_of(a.seg_z[row + k0 + u], part) : 0.0;
                gg[u] = in ? a.seg_g[row + k0 + u] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                if (k0 + u < Km) {
                    reinterpret_cast<double*>(a.cf + row + k0 + u)[part] = c;
                    c = fma(gg[u], c, zz[u]);
                }
            }
        }
    } else {
        double d = 0.0, tot = 0.0;
        for (int k0 = Km - 1; k0 >= 0; k0 -= CH) {
            double xx[CH], hh[CH];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const bool in = k0 - u >= 0;
                xx[u] = in ? part_of(a.seg_x[row + k0 - u], part) : 0.0;
                hh[u] = in ? a.seg_h[row + k0 - u] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                if (k0 - u >= 0) {
                    const int kk = k0 - u;
                    reinterpret_cast<double*>(a.cb + row + kk)[part] = d;
                    if (m == 0) tot += fma(a.sum_h[kk], d, part_of(a.sum_x[kk], part));
                    d = fma(hh[u], d, xx[u]);
                }
            }
        }
        if (m == 0) reinterpret_cast<double*>(a.mu)[part] = tot / a.N;
    }
}

template <int PH>
__global__ void __launch_bounds__(STH) solve_tile_kernel(const SolveArgs a) {
    solve_tile_body<PH>(a, blockIdx.x);
}

template <bool FWD>
__global__ void __launch_bounds__(SCAN_TH) solve_scan_kernel(const SolveArgs a) {
    scan_body<FWD>(a, blockIdx.x * SCAN_TH + threadIdx.x);
}

// Grouped: one grid over several instances (tile counts prefix-summed in offs).
template <int PH>
__global__ void __launch_bounds__(STH) solve_tile_grouped(const SolveArgs* tab, const int* offs, int n, int gate) {
    const int inst = zt_group_find(offs, n, blockIdx.x);
    SolveArgs a = tab[inst];
    a.gate = gate;
    solve_tile_body<PH>(a, blockIdx.x - offs[inst]);
}

// Grouped scans: blockIdx.y is the instance; blocks past an instance's size return.
template <bool FWD>
__global__ void __launch_bounds__(SCAN_TH) solve_scan_grouped(const SolveArgs* tab, int gate) {
    SolveArgs a = tab[blockIdx.y];
    a.gate = gate;
    scan_body<FWD>(a, blockIdx.x * SCAN_TH + threadIdx.x);
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
static int solve_tiles(int N) {
    int tiles = 0;
    for (int b = 0; b * SD < N; ++b) tiles += (N - b * SD + SL - 1) / SL;
    return tiles;
}

static int scan_ctas(int N) { return (2 * N + SCAN_TH - 1) / SCAN_TH; }

// Offset of every diagonal in the diagonal-major layout (each padded to CH entries).
static std::vector<long long> diag_offsets(int N) {
    std::vector<long long> dof((size_t)N + 1);
    long long o = 0;
    for (int m = 0; m < N; ++m) {
        dof[m] = o;
        o += (N - m + CH - 1) / CH * CH;
    }
    dof[N] = o;
    return dof;
}

int zt_solve_create(zt_plan* p) {
    const int N = p->N;
    p->nseg = (N + SL - 1) / SL;
    const size_t ns = (size_t)N * p->nseg;
    const size_t nd = (size_t)diag_offsets(N)[N];
    ZT_CU(ZT_DMALLOC(p->fac_l, nd * sizeof(double), p->mstream));
    ZT_CU(ZT_DMALLOC(p->fac_nd, nd * sizeof(double), p->mstream));
    ZT_CU(ZT_DMALLOC(p->fac_g, nd * sizeof(double), p->mstream));
    ZT_CU(ZT_DMALLOC(p->fac_h, nd * sizeof(double), p->mstream));
    ZT_CU(ZT_DMALLOC(p->dof, ((size_t)N + 1) * sizeof(long long), p->mstream));
    ZT_CU(ZT_DMALLOC(p->seg_z, ns * sizeof(double2), p->mstream));
    ZT_CU(ZT_DMALLOC(p->seg_g, ns * sizeof(double), p->mstream));
    ZT_CU(ZT_DMALLOC(p->seg_x, ns * sizeof(double2), p->mstream));
    ZT_CU(ZT_DMALLOC(p->seg_h, ns * sizeof(double), p->mstream));
    ZT_CU(ZT_DMALLOC(p->carry_f, ns * sizeof(double2), p->mstream));
    ZT_CU(ZT_DMALLOC(p->carry_b, ns * sizeof(double2), p->mstream));
    ZT_CU(ZT_DMALLOC(p->sum_x, (size_t)p->nseg * sizeof(double2), p->mstream));
    ZT_CU(ZT_DMALLOC(p->sum_h, (size_t)p->nseg * sizeof(double), p->mstream));
    ZT_CU(ZT_DMALLOC(p->sol_mu, sizeof(double2), p->mstream));
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
    zt_dfree(p->fac_l, p->mstream);
    zt_dfree(p->fac_nd, p->mstream);
    zt_dfree(p->fac_g, p->mstream);
    zt_dfree(p->fac_h, p->mstream);
    zt_dfree(p->dof, p->mstream);
    zt_dfree(p->seg_z, p->mstream);
    zt_dfree(p->seg_g, p->mstream);
    zt_dfree(p->seg_x, p->mstream);
    zt_dfree(p->seg_h, p->mstream);
    zt_dfree(p->carry_f, p->mstream);
    zt_dfree(p->carry_b, p->mstream);
    zt_dfree(p->sum_x, p->mstream);
    zt_dfree(p->sum_h, p->mstream);
    zt_dfree(p->sol_mu, p->mstream);
}

size_t zt_solve_bytes(int N) {
    const size_t nseg = (size_t)(N + SL - 1) / SL, ns = (size_t)N * nseg;
    const size_t nd = (size_t)diag_offsets(N)[N];
    return 4 * nd * 8 + ((size_t)N + 1) * 8 + ns * (16 + 8 + 16 + 8 + 16 + 16) + nseg * 24 + 16;
}

// Diagonal m in diagonal-major order, and the products of its factors within
// each segment in the order the recurrences apply them:  G_i = prod_{j=i0..i}
// (-l_j) (forward) and H_i = prod_{j=i+1..i1} (-l_j) (backward; l at i1 = n
// counts as 0).
static void diagonal_data(int N, int m, int K, const long long* dof, const double* l_tri, const double* nd_tri,
                          double* L, double* ND, double* G, double* H, double* sg, double* sh, double* shsum) {
    const int n = N - m;
    double* Lm = L + dof[m];
    for (int i = 0; i < n; ++i) {
        const size_t at = zt_tri(i + m, i);
        Lm[i] = l_tri[at];
        ND[dof[m] + i] = nd_tri[at];
    }
    for (int k = 0; k * SL < n; ++k) {
        const int i0 = k * SL, i1 = i0 + SL < n ? i0 + SL : n;
        double g = 1.0;
        for (int i = i0; i < i1; ++i) {
            g *= -Lm[i];
            G[dof[m] + i] = g;
        }
        sg[(size_t)m * K + k] = g;
        double h = (i1 < n) ? -Lm[i1] : 0.0, hs = 0.0;
        for (int i = i1 - 1; i >= i0; --i) {
            if (i < i1 - 1) h *= -Lm[i + 1];
            H[dof[m] + i] = h;
            hs += h;
        }
        sh[(size_t)m * K + k] = h;
        if (m == 0) shsum[k] = hs;
    }
}

int zt_solve_upload_factors(zt_plan* p, const double* host_l, const double* host_nd) {
    const int N = p->N, K = p->nseg;
    const size_t nk = (size_t)N * K;
    std::vector<long long> dof = diag_offsets(N);
    const size_t nd = (size_t)dof[N];
    std::vector<double> L, ND, G, H, sg, sh, shsum;
    try {   // zero padding past each diagonal's end is read (and ignored) by the kernels
        L.assign(nd, 0.0);
        ND.assign(nd, 0.0);
        G.assign(nd, 0.0);
        H.assign(nd, 0.0);
        sg.assign(nk, 0.0);
        sh.assign(nk, 0.0);
        shsum.assign((size_t)K, 0.0);
    } catch (...) {
        return zt_fail(ZT_ENOMEM, "host allocation for the solve factors failed");
    }
    unsigned nt = std::thread::hardware_concurrency();
    nt = nt == 0 ? 1 : (nt > 16 ? 16 : nt);
    if ((long long)N * N < 1 << 20) nt = 1;
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            for (int m = (int)t; m < N; m += (int)nt)
                diagonal_data(N, m, K, dof.data(), host_l, host_nd, L.data(), ND.data(), G.data(), H.data(),
                              sg.data(), sh.data(), shsum.data());
        });
    for (auto& x : th) x.join();
    cudaStream_t cs = p->mstream;
    cudaMemcpyAsync(p->fac_l, L.data(), nd * sizeof(double), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(p->fac_nd, ND.data(), nd * sizeof(double), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(p->fac_g, G.data(), nd * sizeof(double), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(p->fac_h, H.data(), nd * sizeof(double), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(p->dof, dof.data(), dof.size() * sizeof(long long), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(p->seg_g, sg.data(), nk * sizeof(double), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(p->seg_h, sh.data(), nk * sizeof(double), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(p->sum_h, shsum.data(), (size_t)K * sizeof(double), cudaMemcpyHostToDevice, cs);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);   // host vectors go out of scope
    if (e != cudaSuccess) return zt_cuda_check(e, "solve factor upload");
    return ZT_OK;
}

int zt_solve_ctas(int N) { return solve_tiles(N); }

int zt_solve_args(zt_plan* p, const double2* W, double2* P, SolveArgs* out) {
    SolveArgs& a = *out;
    a.W = W;
    a.P = P;
    a.fl = p->fac_l;
    a.fnd = p->fac_nd;
    a.fg = p->fac_g;
    a.fh = p->fac_h;
    a.dof = p->dof;
    a.seg_z = p->seg_z;
    a.seg_g = p->seg_g;
    a.seg_x = p->seg_x;
    a.seg_h = p->seg_h;
    a.cf = p->carry_f;
    a.cb = p->carry_b;
    a.sum_x = p->sum_x;
    a.sum_h = p->sum_h;
    a.mu = p->sol_mu;
    a.N = p->N;
    a.K = p->nseg;
    a.st = p->state;
    a.gate = ZT_GATE_NONE;
    return ZT_OK;
}

int zt_solve_grouped(const SolveArgs* tab, const int* offs, int n, int total, int maxN, cudaStream_t s, int gate) {
    const dim3 sg((unsigned)scan_ctas(maxN), (unsigned)n);
    solve_tile_grouped<F1><<<total, STH, TILE_SMEM, s>>>(tab, offs, n, gate);
    solve_scan_grouped<true><<<sg, SCAN_TH, 0, s>>>(tab, gate);
    solve_tile_grouped<B1><<<total, STH, TILE_SMEM, s>>>(tab, offs, n, gate);
    solve_scan_grouped<false><<<sg, SCAN_TH, 0, s>>>(tab, gate);
    solve_tile_grouped<B3><<<total, STH, TILE_SMEM, s>>>(tab, offs, n, gate);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "solve_tile_grouped");
    return ZT_OK;
}

int zt_launch_stream_solve(zt_plan* p, const double2* W, double2* P, cudaStream_t s, int gate) {
    const int N = p->N;
    SolveArgs a;
    zt_solve_args(p, W, P, &a);
    a.gate = gate;
    const int tiles = solve_tiles(N);
    const double bytes = 8.0 * N * (N + 1.0) + 16.0 * N * N;
    const int t = zt_timer_begin(p, ZT_KERNEL_SOLVE, bytes, bytes, s);
    solve_tile_kernel<F1><<<tiles, STH, TILE_SMEM, s>>>(a);
    solve_scan_kernel<true><<<scan_ctas(N), SCAN_TH, 0, s>>>(a);
    solve_tile_kernel<B1><<<tiles, STH, TILE_SMEM, s>>>(a);
    solve_scan_kernel<false><<<scan_ctas(N), SCAN_TH, 0, s>>>(a);
    solve_tile_kernel<B3><<<tiles, STH, TILE_SMEM, s>>>(a);
    zt_timer_end(p, t, s);
    p->launches += ZT_SOLVE_LAUNCHES;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "solve_tile_kernel");
    return ZT_OK;
}
