// Quantised spherical-harmonic basis (Sec. 3.2, Eqs. 10-12).
//
// T^_lm with m >= 0 lies on the m-th (lower) diagonal of an N x N matrix:
// its entries there form the unit eigenvector of the tridiagonal block
// -Delta^m (Eq. 13) for the eigenvalue l(l+1), l = m .. N-1
// (Eq. 12), and T^_{l,-m} = (-1)^m T^_lm^T.  The sign follows Eq. 11:
// the last entry of the diagonal carries (-1)^m (its Wigner 3j symbol has a
// stretched column).
//
// Eigenvectors, one thread per (m, l <= lmax): twisted factorization of
// -Delta^m - l(l+1) I at the exact eigenvalue -- forward pivots D+,
// backward pivots D-, twist index k = argmin |gamma_k| with gamma_k = D+_k +
// D-_k - (a_k - lambda) -- then x_k = 1 and the two outward recurrences
// x_i = -(b_i / D+_i) x_{i+1} (i < k), x_i = -(b_{i-1} / D-_i) x_{i-1} (i > k);
// a zero pivot marks a zero entry (the persymmetric blocks have them), and
// the step across it uses the three-term relation.  The global sign is fixed
// at x_k by the backward three-term recurrence from the last entry (-1)^m,
// which grows from that end into the bulk (the end entries themselves can be
// below double precision).
//
// W = sum_lm i omega_lm T^_lm (Eq. 10) is banded (|m| <= lmax): one thread per
// band element sums over l.  omega_lm = -i tr(T^_lm^T W) (orthonormal basis):
// one warp per (l, m) reduces along its diagonal in a fixed order.
#include <cmath>
#include <vector>

#include "zt_internal.h"

struct zt_basis {
    int N = 0, lmax = 0, npairs = 0;
    long long nvec = 0;                // doubles in vec
    double* vec = nullptr;             // v_lm, pair p at voff[p], N - m entries
    long long* voff = nullptr;         // [npairs]
    cudaStream_t own = nullptr;        // private stream for allocation and frees (no plan is kept)
    cudaEvent_t last_use = nullptr;    // last launch that reads vec (frees wait for it)
    std::vector<long long> hoff;       // host copy of voff
};

namespace {
constexpr int BV_TH = 64;
constexpr int WO_TH = 256;
constexpr int OW_WARPS = 8;

__device__ __forceinline__ int pair_index(int l, int m, int lmax) {   // m = 0..lmax, l = m..lmax
    return m * (lmax + 1) - m * (m - 1) / 2 + (l - m);
}
}  // namespace

__global__ void __launch_bounds__(BV_TH) basis_vectors_kernel(const double* __restrict__ la,
                                                              const double* __restrict__ lb, int N,
                                                              const int* __restrict__ pl, const int* __restrict__ pm,
                                                              const long long* __restrict__ voff, double* vec,
                                                              double* scr, int npairs) {
    const int p = blockIdx.x * BV_TH + threadIdx.x;
    if (p >= npairs) return;
    const int l = pl[p], m = pm[p], n = N - m;
    double* x = vec + voff[p];
    double* dm = scr + voff[p];
    const double lam = (double)l * (l + 1);
    auto A = [&](int i) { return la[zt_tri(i + m, i)] - lam; };   // diagonal of -Delta^m - lambda I
    auto Bo = [&](int i) { return lb[zt_tri(i + m, i)]; };        // couples positions i and i + 1 (< 0)
    if (n == 1) {
        x[0] = (m & 1) ? -1.0 : 1.0;
        return;
    }
    // forward pivots into x, backward pivots into dm; twist index
    double dp = A(0);
    x[0] = dp;
    for (int i = 1; i < n; ++i) {
        const double b = Bo(i - 1);
        dp = (dp != 0.0) ? A(i) - b * b / dp : -INFINITY;   // D+_{i-1} = 0: x_i = 0 exactly
        x[i] = dp;
    }
    double dmi = A(n - 1);
    dm[n - 1] = dmi;
    int k = n - 1;
    double gbest = fabs(x[n - 1]);
    for (int i = n - 2; i >= 0; --i) {
        const double b = Bo(i);
        dmi = (dmi != 0.0) ? A(i) - b * b / dmi : -INFINITY;
        dm[i] = dmi;
        const double g = fabs(x[i] + dmi - A(i));
        if (g < gbest) {
            gbest = g;
            k = i;
        }
    }
    // outward from x_k = 1 (x[i] still holds D+_i for i < k while it is read)
    double x1 = 1.0, x2 = 0.0;   // x_{i+1}, x_{i+2}
    for (int i = k - 1; i >= 0; --i) {
        const double piv = x[i];
        double v;
        if (piv != 0.0)   // an infinite pivot gives the zero entry after a zero pivot
            v = -(Bo(i) / piv) * x1;
        else   // x_{i+1} = 0: row i + 1 gives b_i x_i + b_{i+1} x_{i+2} = 0
            v = -(Bo(i + 1) / Bo(i)) * x2;
        x[i] = v;
        x2 = x1;
        x1 = v;
    }
    x[k] = 1.0;
    x1 = 1.0;
    x2 = 0.0;   // x_{i-1}, x_{i-2}
    for (int i = k + 1; i < n; ++i) {
        const double piv = dm[i];
        double v;
        if (piv != 0.0)   // an infinite pivot gives the zero entry after a zero pivot
            v = -(Bo(i - 1) / piv) * x1;
        else   // x_{i-1} = 0: row i - 1 gives b_{i-2} x_{i-2} + b_{i-1} x_i = 0 (no x_{-1})
            v = (i >= 2) ? -(Bo(i - 2) / Bo(i - 1)) * x2 : 0.0;
        x[i] = v;
        x2 = x1;
        x1 = v;
    }
    // sign at k from the backward three-term recurrence, y[n-1] = (-1)^m
    double y1 = (m & 1) ? -1.0 : 1.0, y0 = 0.0;   // y_i, y_{i+1}
    for (int i = n - 1; i > k; --i) {
        const double nxt = -(A(i) * y1 + (i + 1 < n ? Bo(i) * y0 : 0.0)) / Bo(i - 1);
        y0 = y1;
        y1 = nxt;
        const double big = fmax(fabs(y0), fabs(y1));
        if (big > 1e100) {
            y0 /= big;
            y1 /= big;
        }
    }
    double ss = 0.0;
    for (int i = 0; i < n; ++i) ss += x[i] * x[i];
    double sc = 1.0 / sqrt(ss);
    if (y1 < 0.0) sc = -sc;   // x_k = 1 > 0
    for (int i = 0; i < n; ++i) x[i] *= sc;
}

// W on the band |d| <= lmax: element (i + d, i) for d >= 0, (i, i - d) for d < 0.
__global__ void __launch_bounds__(WO_TH) w_from_omega_kernel(const double2* __restrict__ om,
                                                             const double* __restrict__ vec,
                                                             const long long* __restrict__ voff, int N, int lmax,
                                                             double2* __restrict__ W) {
    const int d = (int)blockIdx.y - lmax;
    const int m = d < 0 ? -d : d;
    const int i = blockIdx.x * WO_TH + threadIdx.x;
    if (i >= N - m) return;
    const double sgn = (d < 0 && (m & 1)) ? -1.0 : 1.0;   // T^_{l,-m} = (-1)^m T^_lm^T
    double re = 0.0, im = 0.0;
    for (int l = m; l <= lmax; ++l) {
        const double2 o = om[l * l + l + d];
        const double v = sgn * vec[voff[pair_index(l, m, lmax)] + i];
        re -= o.y * v;   // i omega v
        im += o.x * v;
    }
    const size_t r = d >= 0 ? (size_t)(i + m) : (size_t)i, c = d >= 0 ? (size_t)i : (size_t)(i + m);
    W[r * N + c] = make_double2(re, im);
}

// omega_{l,d} = -i sum_i T^_{l,d}(entry) W(entry), one warp per (l, d), |d| <= l.
__global__ void omega_from_w_kernel(const double2* __restrict__ W, const double* __restrict__ vec,
                                    const long long* __restrict__ voff, int N, int lmax, double2* __restrict__ om) {
    const int q = blockIdx.x * OW_WARPS + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const int nq = (lmax + 1) * (lmax + 1);
    if (q >= nq) return;
    int l = 0;
    while ((l + 1) * (l + 1) <= q) ++l;
    const int d = q - l * l - l, m = d < 0 ? -d : d, n = N - m;
    const double* v = vec + voff[pair_index(l, m, lmax)];
    double sr = 0.0, si = 0.0;
    for (int i = lane; i < n; i += 32) {
        const size_t r = d >= 0 ? (size_t)(i + m) : (size_t)i, c = d >= 0 ? (size_t)i : (size_t)(i + m);
        const double2 w = W[r * N + c];
        sr += v[i] * w.x;
        si += v[i] * w.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
        const double sgn = (d < 0 && (m & 1)) ? -1.0 : 1.0;
        om[q] = make_double2(sgn * si, -sgn * sr);   // -i (sr + i si)
    }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
extern "C" void zt_basis_destroy(zt_basis* b) {
    if (!b) return;
    if (b->own) {
        if (b->last_use) cudaStreamWaitEvent(b->own, b->last_use, 0);   // frees after the last reader
        zt_dfree(b->vec, b->own);
        zt_dfree(b->voff, b->own);
        cudaStreamSynchronize(b->own);
        cudaStreamDestroy(b->own);
    }
    if (b->last_use) cudaEventDestroy(b->last_use);
    delete b;
}

extern "C" int zt_basis_create(zt_plan* p, int lmax, zt_basis** out) {
    if (!out) return zt_fail(ZT_EINVAL, "zt_basis_create: out is NULL");
    *out = nullptr;
    if (!p) return zt_fail(ZT_EINVAL, "zt_basis_create: plan is NULL");
    if (lmax < 0 || lmax > p->N - 1) return zt_fail(ZT_EINVAL, "zt_basis_create: lmax=%d outside [0, N-1]", lmax);
    zt_basis* b = new (std::nothrow) zt_basis();
    if (!b) return zt_fail(ZT_ENOMEM, "zt_basis_create: host allocation failed");
    b->N = p->N;
    b->lmax = lmax;
    std::vector<int> hl, hm;
    long long off = 0;
    for (int m = 0; m <= lmax; ++m)
        for (int l = m; l <= lmax; ++l) {
            hl.push_back(l);
            hm.push_back(m);
            b->hoff.push_back(off);
            off += p->N - m;
        }
    b->npairs = (int)hl.size();
    b->nvec = off;
    double* scr = nullptr;   // backward pivots, creation only
    int *pl = nullptr, *pm = nullptr;
    auto fail = [&](int rc) {
        if (b->own) {
            zt_dfree(scr, b->own);
            zt_dfree(pl, b->own);
            zt_dfree(pm, b->own);
        }
        zt_basis_destroy(b);
        return rc;
    };
    cudaError_t e;
    if ((e = zt_setup_stream(&b->own)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->last_use, cudaEventDisableTiming)) != cudaSuccess)
        return fail(zt_cuda_check(e, "zt_basis_create (stream)"));
    cudaStream_t cs = b->own;
    if ((e = ZT_DMALLOC(b->vec, (size_t)off * sizeof(double), cs)) != cudaSuccess ||
        (e = ZT_DMALLOC(scr, (size_t)off * sizeof(double), cs)) != cudaSuccess ||
        (e = ZT_DMALLOC(b->voff, (size_t)b->npairs * sizeof(long long), cs)) != cudaSuccess ||
        (e = ZT_DMALLOC(pl, (size_t)b->npairs * sizeof(int), cs)) != cudaSuccess ||
        (e = ZT_DMALLOC(pm, (size_t)b->npairs * sizeof(int), cs)) != cudaSuccess)
        return fail(zt_cuda_check(e, "zt_basis_create (allocation)"));
    if ((e = cudaStreamSynchronize(p->mstream)) != cudaSuccess)   // the plan's Laplacian is uploaded
        return fail(zt_cuda_check(e, "zt_basis_create (plan stream)"));
    cudaMemcpyAsync(b->voff, b->hoff.data(), b->hoff.size() * sizeof(long long), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(pl, hl.data(), hl.size() * sizeof(int), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(pm, hm.data(), hm.size() * sizeof(int), cudaMemcpyHostToDevice, cs);
    basis_vectors_kernel<<<(b->npairs + BV_TH - 1) / BV_TH, BV_TH, 0, cs>>>(p->lap_a, p->lap_b, p->N, pl, pm,
                                                                        b->voff, b->vec, scr, b->npairs);
    e = cudaGetLastError();
    zt_dfree(scr, cs);
    zt_dfree(pl, cs);
    zt_dfree(pm, cs);
    scr = nullptr;
    pl = pm = nullptr;
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);   // host vectors go out of scope
    if (e != cudaSuccess) return fail(zt_cuda_check(e, "zt_basis_create"));
    *out = b;
    return ZT_OK;
}

extern "C" int zt_basis_vector(zt_basis* b, int l, int m, double* out) {
    if (!b || !out) return zt_fail(ZT_EINVAL, "zt_basis_vector: NULL argument");
    if (m < 0 || m > l || l > b->lmax) return zt_fail(ZT_EINVAL, "zt_basis_vector: need 0 <= m <= l <= lmax");
    const int p = m * (b->lmax + 1) - m * (m - 1) / 2 + (l - m);
    ZT_CU(cudaMemcpy(out, b->vec + b->hoff[p], (size_t)(b->N - m) * sizeof(double), cudaMemcpyDeviceToHost));
    return ZT_OK;
}

static int check_dev(const void* q, const char* what) {
    if (!q) return zt_fail(ZT_EINVAL, "%s is NULL", what);
    if (((uintptr_t)q) & 15u) return zt_fail(ZT_EINVAL, "%s is not 16-byte aligned", what);
    return ZT_OK;
}

extern "C" int zeitlin_w_from_omega(zt_basis* b, const double* omega, double* W, void* stream) {
    if (!b) return zt_fail(ZT_EINVAL, "basis is NULL");
    int rc;
    if ((rc = check_dev(omega, "omega")) || (rc = check_dev(W, "W"))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = (size_t)b->N;
    ZT_CU(cudaMemsetAsync(W, 0, N * N * sizeof(double2), s));
    const dim3 grid((unsigned)((b->N + WO_TH - 1) / WO_TH), (unsigned)(2 * b->lmax + 1));
    w_from_omega_kernel<<<grid, WO_TH, 0, s>>>((const double2*)omega, b->vec, b->voff, b->N, b->lmax, (double2*)W);
    ZT_CU(cudaGetLastError());
    cudaEventRecord(b->last_use, s);
    return ZT_OK;
}

extern "C" int zeitlin_omega_from_w(zt_basis* b, const double* W, double* omega, void* stream) {
    if (!b) return zt_fail(ZT_EINVAL, "basis is NULL");
    int rc;
    if ((rc = check_dev(omega, "omega")) || (rc = check_dev(W, "W"))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int nq = (b->lmax + 1) * (b->lmax + 1);
    omega_from_w_kernel<<<(nq + OW_WARPS - 1) / OW_WARPS, OW_WARPS * 32, 0, s>>>(
        (const double2*)W, b->vec, b->voff, b->N, b->lmax, (double2*)omega);
    ZT_CU(cudaGetLastError());
    cudaEventRecord(b->last_use, s);
    return ZT_OK;
}
