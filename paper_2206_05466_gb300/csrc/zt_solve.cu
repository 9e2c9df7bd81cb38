// Stream solve P = Delta_N^{-1} W (Sec. 3.3, Eq. 14), by bands of diagonals.
//
// Diagonal m (0 <= m < N) of the lower triangle holds the n = N-m unknowns of
// the tridiagonal system T_m x = -w (T_m = -Delta^m, Eq. 13), solved with the
// plan's LDL^T factors:
//     forward   z_i = w_i + nl_i z_{i-1}                 (nl_i = -l_i, l_0 = 0)
//     backward  x_i = nd_i z_i + nl_{i+1} x_{i+1}         (nd_i = -1/d_i)
// The device holds nl, not l: on GB300 a stand-alone FP64 negation is an
// instruction of the narrow FP64 pipe, and the sweeps are bound by that pipe.
//
// Layout of the work.  A band is 32 consecutive diagonals m0 .. m0+31, one per
// lane of a warp.  In row r the band's elements (r, r-m), m in the band, are
// 32 adjacent entries of that row: one 512-byte run of W or P, so a warp reads
// or writes a whole row of its band in one coalesced access, and the
// per-element factors (packed lower-triangular, row-major, as the pairs
// (-l, nd) and (F, H): one 16-byte load each) likewise.  A warp
// works on a segment of SL = 16 rows of its band; for lane t (diagonal m0 + t)
// that is the positions [16k - t, 16k + 16 - t) of its diagonal (empty for the
// first segment of lanes t >= 16).
//
// Both recurrences are linear, so each segment is swept from zero inflows and
// corrected afterwards.  With c the true z just before the segment and d the
// true x just after it,
//     z_i = z0_i + G_i c,              G_i = prod_{j = s0..i} (-l_j)
//     x_i = x0_i + F_i c + H_i d,
// where x0 is the backward sweep of nd z0 from a zero right inflow, F the
// backward sweep of nd G (the segment's response to c) and H_i = prod_{j =
// i+1..s1} (-l_j) (its response to d).  G, F and H depend only on the
// factors: the plan computes them once.  Three launches:
//   FB  per (band, segment) warp: forward sweep z0 (kept in shared memory),
//       then backward sweep x0, parked in the lower triangle of P; the
//       segment's last z0 and first x0 go to small [K][N] arrays;
//   S   one warp per diagonal: the forward inflows c_k from the segments'
//       end values, then the backward inflows d_k, each a first-order linear
//       recurrence over k scanned in parallel across the lanes; for m = 0 also
//       the mean of the solution;
//   C   per (band, segment) warp: x = x0 + F c + H d, written to the lower
//       triangle row by row and, as -conj, to the upper triangle (the mirror
//       of a band segment is a set of partial row runs, written from shared
//       memory).
// FB and C issue every load of a segment before its first dependent
// operation: the 16 rows of W (FB) or x0 (C) go to the warp's shared memory
// by asynchronous copies, the factor pairs to registers (which is what bounds
// the kernels to 16 warps per SM).
// FP64 work: 3 + 2 fused operations per real component and element.
//
// The singular m = 0 block (the l = 0 mode): the mean of its right-hand side
// is removed before the forward sweep (band-0 warps reduce diagonal 0 of W
// while their copies are in flight), the leading N-1 equations are solved with x_{N-1} = 0 (the factors
// of the dropped row are zero), and the mean of the solution is removed in C.
#include <thread>
#include <vector>

#include "zt_internal.h"

namespace {
constexpr int BW = 32;            // diagonals per band (lanes of a warp)
constexpr int SL = 16;            // rows per segment: 8 KB of shared memory per warp
constexpr int SPB = BW / SL;      // segments per 32 rows of a band
static_assert(BW % SL == 0, "a band's 32-row blocks split into whole segments");
constexpr int WPC = 4;            // warps per CTA; 4 CTAs per SM (the 2 x 16 factors of a lane's segment
                                  // are held in registers)
constexpr size_t WARP_SMEM = (size_t)SL * BW * sizeof(double2);
constexpr size_t CTA_SMEM = WPC * WARP_SMEM;
constexpr int SCAN_TH = 128;   // threads of a scan CTA: one warp per diagonal

// 16-byte asynchronous copy global -> shared (both addresses 16-byte aligned:
// W and P are checked on entry, the staging rows are 16-byte slots).
__device__ __forceinline__ void zt_cp_async16(void* smem_dst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void zt_cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__host__ __device__ inline int nbands(int N) { return (N + BW - 1) / BW; }
// Segments of band b: SPB (nbands - b), the rows m0 = 32 b .. 32 nbands - 1 in
// blocks of SL (trailing ones may lie past row N - 1; for lane t >= SL the
// first segment holds no position of its diagonal).  Band 0 has nseg(N).
__host__ __device__ inline int nseg(int N) { return SPB * nbands(N); }
__host__ __device__ inline int band_segs(int N, int b) { return SPB * (nbands(N) - b); }
__host__ __device__ inline int items(int N) {   // (band, segment) pairs
    const int nb = nbands(N);
    return SPB * (nb * (nb + 1) / 2);
}

// Work item q -> (band b, segment k).  Items are enumerated band by band from
// the last band (SPB segments) to band 0 (nseg segments): band nb - 1 - r
// starts at item SPB r (r + 1) / 2.
__device__ __forceinline__ void item_of(int q, int N, int& b, int& k) {
    int r = (int)((sqrtf(8.0f * (float)(q / SPB) + 1.0f) - 1.0f) * 0.5f);
    while (r > 0 && SPB * (r * (r + 1) / 2) > q) --r;
    while (SPB * ((r + 1) * (r + 2) / 2) <= q) ++r;
    k = q - SPB * (r * (r + 1) / 2);
    b = nbands(N) - 1 - r;
}
}  // namespace

// ---- FB: local forward and backward sweeps of one band segment ----
// B0: band 0, which holds the singular m = 0 block.  The two cases are separate
// instantiations: with a runtime test the compiler executes the band-0 adds
// (of zeros) in every band, and on GB300 each is an issue slot of the FP64 pipe.
template <bool B0>
__device__ __forceinline__ void solve_fb_band(const SolveArgs& a, int b, int k, double2* zs) {
    const int N = a.N, lane = threadIdx.x & 31;
    const int m0 = b * BW, R0 = m0 + k * SL, R1 = min(R0 + SL, N);
    const int m = m0 + lane;
    const bool valid = m < N;
    const double2* __restrict__ W = a.W;
    const double2* __restrict__ fln = a.fln;

    // Every load of the segment is issued before the first dependent operation:
    // W's rows go to shared memory by asynchronous copies (zs[row][lane], later
    // overwritten by z0), the factor pairs (-l, nd) to registers.
    double nl[SL], nd[SL];
#pragma unroll
    for (int u = 0; u < SL; ++u) {
        const int r = R0 + u;
        if (valid && r < R1 && r >= m) {
            zt_cp_async16(zs + u * BW + lane, W + (size_t)r * N + (r - m));
            const double2 q = __ldg(fln + zt_tri(r, r - m));
            nl[u] = q.x;
            nd[u] = q.y;
        } else {
            nl[u] = nd[u] = 0.0;
        }
    }

    // m = 0: mean of the right-hand side (diagonal 0 of W), reduced by the warp
    // while the copies are in flight
    double mur = 0.0, mui = 0.0;
    if (B0) {   // eight strided loads in flight per lane
        constexpr int UR = 8;
        for (int i0 = lane; i0 < N; i0 += 32 * UR) {
            double2 v[UR];
#pragma unroll
            for (int u = 0; u < UR; ++u) {
                const int i = i0 + 32 * u;
                v[u] = i < N ? W[(size_t)i * N + i] : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int u = 0; u < UR; ++u) {
                mur += v[u].x;
                mui += v[u].y;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            mur += __shfl_xor_sync(0xffffffffu, mur, o);
            mui += __shfl_xor_sync(0xffffffffu, mui, o);
        }
        mur = m == 0 ? mur / N : 0.0;
        mui = m == 0 ? mui / N : 0.0;
    }
    zt_cp_async_wait_all();   // each lane reads back only the rows it copied

    // forward sweep from a zero inflow, z0 in place of w
    double zr = 0.0, zi = 0.0;
#pragma unroll
    for (int u = 0; u < SL; ++u) {
        const int r = R0 + u;
        if (valid && r < R1 && r >= m) {
            double2 w = zs[u * BW + lane];
            if (B0) {
                w.x -= mur;
                w.y -= mui;
            }
            zr = fma(nl[u], zr, w.x);
            zi = fma(nl[u], zi, w.y);
            zs[u * BW + lane] = make_double2(zr, zi);
        }
    }
    if (valid) a.seg_z[(size_t)k * N + m] = make_double2(zr, zi);   // the last row of the segment is active

    // backward sweep of nd z0 from a zero right inflow
    double xr = 0.0, xi = 0.0, lnext = 0.0, sxr = 0.0, sxi = 0.0;
#pragma unroll
    for (int u = SL - 1; u >= 0; --u) {
        const int r = R0 + u;
        if (valid && r < R1 && r >= m) {
            const double2 z = zs[u * BW + lane];
            xr = fma(lnext, xr, nd[u] * z.x);
            xi = fma(lnext, xi, nd[u] * z.y);
            a.P[(size_t)r * N + (r - m)] = make_double2(xr, xi);
            if (B0) {   // segment sums for the m = 0 mean
                sxr += xr;
                sxi += xi;
            }
            lnext = nl[u];
        }
    }
    if (valid) a.seg_x[(size_t)k * N + m] = make_double2(xr, xi);   // x0 at the segment's first position
    if (B0 && m == 0) a.sum_x[k] = make_double2(sxr, sxi);
}

// FB takes the items in reverse order, band 0 first: its warps also reduce
// diagonal 0 for the m = 0 mean, so they must not be the last to start.
__device__ __forceinline__ void solve_fb_body(const SolveArgs& a, int q, double2* zs) {
    if (zt_gate_skip(a.st, a.gate)) return;
    int b, k;
    item_of(items(a.N) - 1 - q, a.N, b, k);
    if (b == 0)
        solve_fb_band<true>(a, b, k, zs);
    else
        solve_fb_band<false>(a, b, k, zs);
}

// ---- S: inflows of every segment of one diagonal, one warp per diagonal ----
//   forward:  c_0 = 0,  c_{k+1} = G_end(k) c_k + z0_end(k)
//   backward: d_{K-1} = 0,  d_{k-1} = x0_start(k) + F_start(k) c_k + H_start(k) d_k
// Both are first-order linear recurrences, so the warp scans them in parallel:
// lane j owns a run of at most PM consecutive segments and composes their
// affine maps (v -> A v + B), a shuffle scan composes the runs (forward from
// lane 0, backward from lane 31), and each lane replays its run from the
// inflow it receives.  All of a run's inputs are loaded at once into
// registers, so the whole scan costs one round trip to memory.  For m = 0 also
// the mean of the solution, sum_k (sum x0 + c_k sum F + d_k sum H) / N,
// reduced over the lanes in a fixed order.
template <int PM>
__device__ __forceinline__ void solve_scan_run(const SolveArgs& a, int m, int k0, int k1) {
    const int N = a.N, lane = threadIdx.x & 31;
    constexpr unsigned FULL = 0xffffffffu;
    double g[PM], h[PM], f[PM];
    double2 z[PM], x0[PM], c[PM];
#pragma unroll
    for (int u = 0; u < PM; ++u) {
        const int k = k0 + u;
        if (k < k1) {
            const size_t e = (size_t)k * N + m;
            g[u] = __ldg(a.seg_g + e);
            h[u] = __ldg(a.seg_h + e);
            f[u] = __ldg(a.seg_f + e);
            z[u] = __ldg(a.seg_z + e);
            x0[u] = __ldg(a.seg_x + e);
        } else {   // identity maps past the run
            g[u] = h[u] = 1.0;
            f[u] = 0.0;
            z[u] = x0[u] = make_double2(0.0, 0.0);
        }
    }
    // forward: this run's map, then the maps of all runs before it
    double A = 1.0, Br = 0.0, Bi = 0.0;
#pragma unroll
    for (int u = 0; u < PM; ++u) {
        Br = fma(g[u], Br, z[u].x);
        Bi = fma(g[u], Bi, z[u].y);
        A *= g[u];
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double Ap = __shfl_up_sync(FULL, A, o);
        const double Brp = __shfl_up_sync(FULL, Br, o);
        const double Bip = __shfl_up_sync(FULL, Bi, o);
        if (lane >= o) {
            Br = fma(A, Brp, Br);
            Bi = fma(A, Bip, Bi);
            A *= Ap;
        }
    }
    double cr = __shfl_up_sync(FULL, Br, 1), ci = __shfl_up_sync(FULL, Bi, 1);
    if (lane == 0) cr = ci = 0.0;
#pragma unroll
    for (int u = 0; u < PM; ++u) {
        c[u] = make_double2(cr, ci);
        if (k0 + u < k1) a.cf[(size_t)(k0 + u) * N + m] = c[u];
        cr = fma(g[u], cr, z[u].x);
        ci = fma(g[u], ci, z[u].y);
    }
    // backward: d_{k-1} = H_k d_k + E_k with E_k = x0_k + F_k c_k, runs composed from lane 31 down
    double2 E[PM];
    A = 1.0;
    Br = Bi = 0.0;
#pragma unroll
    for (int u = PM - 1; u >= 0; --u) {
        E[u] = make_double2(fma(f[u], c[u].x, x0[u].x), fma(f[u], c[u].y, x0[u].y));
        Br = fma(h[u], Br, E[u].x);
        Bi = fma(h[u], Bi, E[u].y);
        A *= h[u];
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double Ap = __shfl_down_sync(FULL, A, o);
        const double Brp = __shfl_down_sync(FULL, Br, o);
        const double Bip = __shfl_down_sync(FULL, Bi, o);
        if (lane + o < 32) {
            Br = fma(A, Brp, Br);
            Bi = fma(A, Bip, Bi);
            A *= Ap;
        }
    }
    double dr = __shfl_down_sync(FULL, Br, 1), di = __shfl_down_sync(FULL, Bi, 1);
    if (lane == 31) dr = di = 0.0;
    double tr = 0.0, ti = 0.0;
#pragma unroll
    for (int u = PM - 1; u >= 0; --u) {
        const int k = k0 + u;
        if (k < k1) {
            a.cb[(size_t)k * N + m] = make_double2(dr, di);
            if (m == 0) {
                const double2 sx0 = a.sum_x[k];
                tr += sx0.x + c[u].x * a.sum_f[k] + dr * a.sum_h[k];
                ti += sx0.y + c[u].y * a.sum_f[k] + di * a.sum_h[k];
            }
        }
        dr = fma(h[u], dr, E[u].x);
        di = fma(h[u], di, E[u].y);
    }
    if (m == 0) {   // warp-uniform
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tr += __shfl_xor_sync(FULL, tr, o);
            ti += __shfl_xor_sync(FULL, ti, o);
        }
        if (lane == 0) *a.mu = make_double2(tr / N, ti / N);
    }
}

// The same scan for runs longer than a few segments (N > 4096): the run's
// values are loaded again where they are needed instead of held in registers.
__device__ __noinline__ void solve_scan_long(const SolveArgs& a, int m, int k0, int k1) {
    const int N = a.N, lane = threadIdx.x & 31;
    constexpr unsigned FULL = 0xffffffffu;
    double A = 1.0, Br = 0.0, Bi = 0.0;
    for (int k = k0; k < k1; ++k) {
        const size_t e = (size_t)k * N + m;
        const double g = __ldg(a.seg_g + e);
        const double2 z = __ldg(a.seg_z + e);
        Br = fma(g, Br, z.x);
        Bi = fma(g, Bi, z.y);
        A *= g;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double Ap = __shfl_up_sync(FULL, A, o);
        const double Brp = __shfl_up_sync(FULL, Br, o);
        const double Bip = __shfl_up_sync(FULL, Bi, o);
        if (lane >= o) {
            Br = fma(A, Brp, Br);
            Bi = fma(A, Bip, Bi);
            A *= Ap;
        }
    }
    double cr = __shfl_up_sync(FULL, Br, 1), ci = __shfl_up_sync(FULL, Bi, 1);
    if (lane == 0) cr = ci = 0.0;
    for (int k = k0; k < k1; ++k) {
        const size_t e = (size_t)k * N + m;
        a.cf[e] = make_double2(cr, ci);
        const double g = __ldg(a.seg_g + e);
        const double2 z = __ldg(a.seg_z + e);
        cr = fma(g, cr, z.x);
        ci = fma(g, ci, z.y);
    }
    A = 1.0;
    Br = Bi = 0.0;
    for (int k = k1 - 1; k >= k0; --k) {
        const size_t e = (size_t)k * N + m;
        const double hk = __ldg(a.seg_h + e), fk = __ldg(a.seg_f + e);
        const double2 x0 = __ldg(a.seg_x + e), c = a.cf[e];   // cf: written above by this lane
        Br = fma(hk, Br, fma(fk, c.x, x0.x));
        Bi = fma(hk, Bi, fma(fk, c.y, x0.y));
        A *= hk;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double Ap = __shfl_down_sync(FULL, A, o);
        const double Brp = __shfl_down_sync(FULL, Br, o);
        const double Bip = __shfl_down_sync(FULL, Bi, o);
        if (lane + o < 32) {
            Br = fma(A, Brp, Br);
            Bi = fma(A, Bip, Bi);
            A *= Ap;
        }
    }
    double dr = __shfl_down_sync(FULL, Br, 1), di = __shfl_down_sync(FULL, Bi, 1);
    if (lane == 31) dr = di = 0.0;
    double tr = 0.0, ti = 0.0;
    for (int k = k1 - 1; k >= k0; --k) {
        const size_t e = (size_t)k * N + m;
        a.cb[e] = make_double2(dr, di);
        const double hk = __ldg(a.seg_h + e), fk = __ldg(a.seg_f + e);
        const double2 x0 = __ldg(a.seg_x + e), c = a.cf[e];
        if (m == 0) {
            const double2 sx0 = a.sum_x[k];
            tr += sx0.x + c.x * a.sum_f[k] + dr * a.sum_h[k];
            ti += sx0.y + c.y * a.sum_f[k] + di * a.sum_h[k];
        }
        dr = fma(hk, dr, fma(fk, c.x, x0.x));
        di = fma(hk, di, fma(fk, c.y, x0.y));
    }
    if (m == 0) {   // warp-uniform
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tr += __shfl_xor_sync(FULL, tr, o);
            ti += __shfl_xor_sync(FULL, ti, o);
        }
        if (lane == 0) *a.mu = make_double2(tr / N, ti / N);
    }
}

__device__ __forceinline__ void solve_scan_body(const SolveArgs& a, int m) {
    if (zt_gate_skip(a.st, a.gate)) return;
    const int N = a.N, lane = threadIdx.x & 31;
    if (m >= N) return;   // warp-uniform
    const int Kb = band_segs(N, m / BW);
    const int per = (Kb + 31) / 32;   // warp-uniform
    const int k0 = min(lane * per, Kb), k1 = min(k0 + per, Kb);
    if (per <= 2)
        solve_scan_run<2>(a, m, k0, k1);
    else if (per <= 4)
        solve_scan_run<4>(a, m, k0, k1);
    else if (per <= 8)
        solve_scan_run<8>(a, m, k0, k1);
    else
        solve_scan_long(a, m, k0, k1);   // N > 4096
}

// ---- C: x = x0 + F c + H d; both triangles ----
template <bool B0>
__device__ __forceinline__ void solve_c_band(const SolveArgs& a, int b, int k, double2* xs) {
    const int N = a.N, lane = threadIdx.x & 31;
    const int m0 = b * BW, R0 = m0 + k * SL, R1 = min(R0 + SL, N);
    const int m = m0 + lane;
    const bool valid = m < N;
    double2 c = make_double2(0.0, 0.0), d = c, mm = c;
    if (valid) {
        c = a.cf[(size_t)k * N + m];
        d = a.cb[(size_t)k * N + m];
        if (B0 && m == 0) mm = *a.mu;
    }
    // x0 (parked in P's lower triangle by FB) to shared memory by asynchronous
    // copies, the pairs (F, H) to registers, all rows of the segment at once
    const double2* __restrict__ ffh = a.ffh;
    double f[SL], h[SL];
#pragma unroll
    for (int u = 0; u < SL; ++u) {
        const int r = R0 + u;
        if (valid && r < R1 && r >= m) {
            zt_cp_async16(xs + u * BW + lane, a.P + (size_t)r * N + (r - m));
            const double2 q = __ldg(ffh + zt_tri(r, r - m));
            f[u] = q.x;
            h[u] = q.y;
        } else {
            f[u] = h[u] = 0.0;
        }
    }
    zt_cp_async_wait_all();   // each lane reads back only the rows it copied
#pragma unroll
    for (int u = 0; u < SL; ++u) {
        const int r = R0 + u;
        if (valid && r < R1 && r >= m) {
            const double2 x0 = xs[u * BW + lane];
            double2 x = make_double2(fma(h[u], d.x, fma(f[u], c.x, x0.x)), fma(h[u], d.y, fma(f[u], c.y, x0.y)));
            if (B0) {   // the m = 0 mean (zero on the other lanes)
                x.x -= mm.x;
                x.y -= mm.y;
            }
            a.P[(size_t)r * N + (r - m)] = x;
            xs[u * BW + lane] = x;
        }
    }
    __syncwarp();
    // upper triangle: P[i, i+m] = -conj(P[i+m, i]).  Upper row i = SL k + j holds, for the
    // lanes t with -t <= j <= SL - 1 - t (and i >= 0, row i + m < R1), adjacent columns i + m.
    for (int j = -(BW - 1); j <= SL - 1; ++j) {
        const int i = k * SL + j;       // position along the diagonals (k * SL = R0 - m0)
        const int rr = j + lane;        // row of the segment holding (i + m, i)
        if (valid && m > 0 && i >= 0 && rr >= 0 && rr < SL && R0 + rr < R1) {
            const double2 x = xs[rr * BW + lane];
            a.P[(size_t)i * N + (i + m)] = make_double2(neg(x.x), x.y);
        }
    }
}

__device__ __forceinline__ void solve_c_body(const SolveArgs& a, int q, double2* xs) {
    if (zt_gate_skip(a.st, a.gate)) return;
    int b, k;
    item_of(q, a.N, b, k);
    if (b == 0)
        solve_c_band<true>(a, b, k, xs);
    else
        solve_c_band<false>(a, b, k, xs);
}

// Single-plan launches are sized to the resident CTAs and stride over the
// items, so that no partial last wave of CTAs leaves most SMs idle.  Item
// q goes to warp q / gridDim.x of CTA q % gridDim.x: consecutive items (the
// band-0 items, which also reduce diagonal 0, come first in FB) land on
// different SMs.
__global__ void __launch_bounds__(WPC * 32, 4) solve_fb_kernel(const SolveArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = threadIdx.x >> 5, nq = items(a.N);
    double2* zs = reinterpret_cast<double2*>(smem) + (size_t)w * SL * BW;
    for (int q = w * gridDim.x + blockIdx.x; q < nq; q += gridDim.x * WPC) {
        solve_fb_body(a, q, zs);
        __syncwarp();
    }
}

__global__ void __launch_bounds__(SCAN_TH) solve_scan_kernel(const SolveArgs a) {
    solve_scan_body(a, (blockIdx.x * SCAN_TH + threadIdx.x) >> 5);
}

__global__ void __launch_bounds__(WPC * 32, 4) solve_c_kernel(const SolveArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = threadIdx.x >> 5, nq = items(a.N);
    double2* xs = reinterpret_cast<double2*>(smem) + (size_t)w * SL * BW;
    for (int q = w * gridDim.x + blockIdx.x; q < nq; q += gridDim.x * WPC) {
        solve_c_body(a, q, xs);
        __syncwarp();
    }
}

// Grouped: one grid over several instances (CTA counts prefix-summed in offs).
__global__ void __launch_bounds__(WPC * 32, 4) solve_fb_grouped(const SolveArgs* tab, const int* offs, int n, int gate) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int inst = zt_group_find(offs, n, blockIdx.x);
    SolveArgs a = tab[inst];
    a.gate = gate;
    const int w = threadIdx.x >> 5;
    const int q = (blockIdx.x - offs[inst]) * WPC + w;
    if (q < items(a.N)) solve_fb_body(a, q, reinterpret_cast<double2*>(smem) + (size_t)w * SL * BW);
}

__global__ void __launch_bounds__(WPC * 32, 4) solve_c_grouped(const SolveArgs* tab, const int* offs, int n, int gate) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int inst = zt_group_find(offs, n, blockIdx.x);
    SolveArgs a = tab[inst];
    a.gate = gate;
    const int w = threadIdx.x >> 5;
    const int q = (blockIdx.x - offs[inst]) * WPC + w;
    if (q < items(a.N)) solve_c_body(a, q, reinterpret_cast<double2*>(smem) + (size_t)w * SL * BW);
}

// Grouped scans: blockIdx.y is the instance; blocks past an instance's size return.
__global__ void __launch_bounds__(SCAN_TH) solve_scan_grouped(const SolveArgs* tab, int gate) {
    SolveArgs a = tab[blockIdx.y];
    a.gate = gate;
    solve_scan_body(a, (blockIdx.x * SCAN_TH + threadIdx.x) >> 5);
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
static int solve_ctas(int N) { return (items(N) + WPC - 1) / WPC; }
static int scan_ctas(int N) { return (N * 32 + SCAN_TH - 1) / SCAN_TH; }

int zt_solve_create(zt_plan* p) {
    const int N = p->N;
    p->nseg = nseg(N);
    const size_t ns = (size_t)N * p->nseg, ntri = (size_t)N * (N + 1) / 2;
    cudaStream_t ms = p->mstream;
    ZT_CU(ZT_DMALLOC(p->fac_lnd, ntri * sizeof(double2), ms));
    ZT_CU(ZT_DMALLOC(p->fac_fh, ntri * sizeof(double2), ms));
    ZT_CU(ZT_DMALLOC(p->seg_z, ns * sizeof(double2), ms));
    ZT_CU(ZT_DMALLOC(p->seg_x, ns * sizeof(double2), ms));
    ZT_CU(ZT_DMALLOC(p->seg_g, ns * sizeof(double), ms));
    ZT_CU(ZT_DMALLOC(p->seg_f, ns * sizeof(double), ms));
    ZT_CU(ZT_DMALLOC(p->seg_h, ns * sizeof(double), ms));
    ZT_CU(ZT_DMALLOC(p->carry_f, ns * sizeof(double2), ms));
    ZT_CU(ZT_DMALLOC(p->carry_b, ns * sizeof(double2), ms));
    ZT_CU(ZT_DMALLOC(p->sum_x, (size_t)p->nseg * sizeof(double2), ms));
    ZT_CU(ZT_DMALLOC(p->sum_f, (size_t)p->nseg * sizeof(double), ms));
    ZT_CU(ZT_DMALLOC(p->sum_h, (size_t)p->nseg * sizeof(double), ms));
    ZT_CU(ZT_DMALLOC(p->sol_mu, sizeof(double2), ms));
    if (!zt_attr_needed(ZT_ATTR_SOLVE)) return ZT_OK;
    ZT_CU(cudaFuncSetAttribute(solve_fb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CTA_SMEM));
    ZT_CU(cudaFuncSetAttribute(solve_c_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CTA_SMEM));
    ZT_CU(cudaFuncSetAttribute(solve_fb_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CTA_SMEM));
    ZT_CU(cudaFuncSetAttribute(solve_c_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CTA_SMEM));
    return ZT_OK;
}

// CTAs of a single-plan sweep launch: all resident at once (the smaller of the
// two kernels' residencies), at most one per warp pair of items.
static int solve_grid(int N) {
    static int resident_of[64] = {};   // per device ordinal, filled on first use (benign race)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return solve_ctas(N);
    }
    int& resident = resident_of[dev];
    if (resident == 0) {
        int nsm = 0, b1 = 0, b2 = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, solve_fb_kernel, WPC * 32, CTA_SMEM) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, solve_c_kernel, WPC * 32, CTA_SMEM) != cudaSuccess ||
            nsm <= 0 || b1 <= 0 || b2 <= 0) {
            cudaGetLastError();
            return solve_ctas(N);
        }
        resident = nsm * (b1 < b2 ? b1 : b2);
    }
    const int c = solve_ctas(N);
    return c < resident ? c : resident;
}

void zt_solve_destroy(zt_plan* p) {
    cudaStream_t ms = p->mstream;
    zt_dfree(p->fac_lnd, ms);
    zt_dfree(p->fac_fh, ms);
    zt_dfree(p->seg_z, ms);
    zt_dfree(p->seg_x, ms);
    zt_dfree(p->seg_g, ms);
    zt_dfree(p->seg_f, ms);
    zt_dfree(p->seg_h, ms);
    zt_dfree(p->carry_f, ms);
    zt_dfree(p->carry_b, ms);
    zt_dfree(p->sum_x, ms);
    zt_dfree(p->sum_f, ms);
    zt_dfree(p->sum_h, ms);
    zt_dfree(p->sol_mu, ms);
}

size_t zt_solve_bytes(int N) {
    const size_t K = (size_t)nseg(N), ns = (size_t)N * K, ntri = (size_t)N * (N + 1) / 2;
    return 4 * ntri * 8 + ns * (16 + 16 + 8 + 8 + 8 + 16 + 16) + K * (16 + 8 + 8) + 16;
}

// Segment responses of diagonal m (lane t = m mod 32 of band m / 32): segment k
// covers positions [max(0, 16k - t), min(n, 16k + 16 - t)).  G (forward
// product over the segment), F (backward sweep of nd G, zero right inflow) and
// H (backward sweep of a unit right inflow); per segment G at its last
// position, F and H at its first, and for m = 0 the sums of F and H.
static void diagonal_responses(int N, int m, const double* l_tri, const double* nd_tri, double* F, double* H,
                               double* sg, double* sf, double* sh, double* sumf, double* sumh,
                               std::vector<double>& G) {
    const int n = N - m, t = m % BW, Kb = band_segs(N, m / BW);
    auto at = [&](int i) { return zt_tri(i + m, i); };
    G.resize((size_t)SL);
    for (int k = 0; k < Kb; ++k) {
        const int s0 = k * SL - t > 0 ? k * SL - t : 0;
        const int s1 = k * SL + SL - t < n ? k * SL + SL - t : n;
        double g = 1.0;
        for (int i = s0; i < s1; ++i) {
            g *= -l_tri[at(i)];
            G[(size_t)(i - s0)] = g;
        }
        const size_t e = (size_t)k * N + m;
        sg[e] = g;
        double f = 0.0, h = 0.0, fs = 0.0, hs = 0.0;
        for (int i = s1 - 1; i >= s0; --i) {
            const double nd = nd_tri[at(i)];
            if (i == s1 - 1) {
                f = nd * G[(size_t)(i - s0)];
                h = (s1 < n) ? -l_tri[at(s1)] : 0.0;
            } else {
                const double ln = l_tri[at(i + 1)];
                f = nd * G[(size_t)(i - s0)] - ln * f;
                h = -ln * h;
            }
            F[at(i)] = f;
            H[at(i)] = h;
            fs += f;
            hs += h;
        }
        sf[e] = f;
        sh[e] = s1 > s0 ? h : 1.0;   // an empty segment passes its inflows on unchanged
        if (m == 0) {
            sumf[k] = fs;
            sumh[k] = hs;
        }
    }
}

int zt_solve_upload_factors(zt_plan* p, const double* host_l, const double* host_nd) {
    const int N = p->N, K = p->nseg;
    const size_t ns = (size_t)N * K, ntri = (size_t)N * (N + 1) / 2;
    std::vector<double> F, H, sg, sf, sh, sumf, sumh;
    std::vector<double2> LND, FH;
    try {
        F.assign(ntri, 0.0);
        H.assign(ntri, 0.0);
        LND.resize(ntri);
        FH.resize(ntri);
        sg.assign(ns, 0.0);
        sf.assign(ns, 0.0);
        sh.assign(ns, 0.0);
        sumf.assign((size_t)K, 0.0);
        sumh.assign((size_t)K, 0.0);
    } catch (...) {
        return zt_fail(ZT_ENOMEM, "host allocation for the solve factors failed");
    }
    unsigned nt = std::thread::hardware_concurrency();
    nt = nt == 0 ? 1 : (nt > 16 ? 16 : nt);
    if ((long long)N * N < 1 << 20) nt = 1;
    std::vector<std::thread> th;
    for (unsigned u = 0; u < nt; ++u)
        th.emplace_back([&, u] {
            std::vector<double> G;
            for (int m = (int)u; m < N; m += (int)nt)
                diagonal_responses(N, m, host_l, host_nd, F.data(), H.data(), sg.data(), sf.data(), sh.data(),
                                   sumf.data(), sumh.data(), G);
        });
    for (auto& x : th) x.join();
    cudaStream_t cs = p->mstream;
    for (size_t i = 0; i < ntri; ++i) {
        LND[i] = make_double2(-host_l[i], host_nd[i]);
        FH[i] = make_double2(F[i], H[i]);
    }
    cudaMemcpyAsync(p->fac_lnd, LND.data(), ntri * sizeof(double2), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(p->fac_fh, FH.data(), ntri * sizeof(double2), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(p->seg_g, sg.data(), ns * sizeof(double), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(p->seg_f, sf.data(), ns * sizeof(double), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(p->seg_h, sh.data(), ns * sizeof(double), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(p->sum_f, sumf.data(), (size_t)K * sizeof(double), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(p->sum_h, sumh.data(), (size_t)K * sizeof(double), cudaMemcpyHostToDevice, cs);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);   // host vectors go out of scope
    if (e != cudaSuccess) return zt_cuda_check(e, "solve factor upload");
    return ZT_OK;
}

int zt_solve_ctas(int N) { return solve_ctas(N); }

int zt_solve_args(zt_plan* p, const double2* W, double2* P, SolveArgs* out) {
    SolveArgs& a = *out;
    a.W = W;
    a.P = P;
    a.fln = p->fac_lnd;
    a.ffh = p->fac_fh;
    a.seg_z = p->seg_z;
    a.seg_x = p->seg_x;
    a.seg_g = p->seg_g;
    a.seg_f = p->seg_f;
    a.seg_h = p->seg_h;
    a.cf = p->carry_f;
    a.cb = p->carry_b;
    a.sum_x = p->sum_x;
    a.sum_f = p->sum_f;
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
    solve_fb_grouped<<<total, WPC * 32, CTA_SMEM, s>>>(tab, offs, n, gate);
    solve_scan_grouped<<<sg, SCAN_TH, 0, s>>>(tab, gate);
    solve_c_grouped<<<total, WPC * 32, CTA_SMEM, s>>>(tab, offs, n, gate);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "solve_grouped");
    return ZT_OK;
}

int zt_launch_stream_solve(zt_plan* p, const double2* W, double2* P, cudaStream_t s, int gate) {
    const int N = p->N;
    SolveArgs a;
    zt_solve_args(p, W, P, &a);
    a.gate = gate;
    const int ctas = solve_grid(N);
    const double bytes = 8.0 * N * (N + 1.0) + 16.0 * N * N;
    const int t = zt_timer_begin(p, ZT_KERNEL_SOLVE, bytes, bytes, s);
    solve_fb_kernel<<<ctas, WPC * 32, CTA_SMEM, s>>>(a);
    solve_scan_kernel<<<scan_ctas(N), SCAN_TH, 0, s>>>(a);
    solve_c_kernel<<<ctas, WPC * 32, CTA_SMEM, s>>>(a);
    zt_timer_end(p, t, s);
    p->launches += ZT_SOLVE_LAUNCHES;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "solve kernels");
    return ZT_OK;
}
