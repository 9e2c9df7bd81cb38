// Plan, Laplacian apply, stream solve, fixed-point update/convergence and the
// IsoMP step driver of libzeitlin (GB300, sm_103a).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>

#include "zt_internal.h"

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

constexpr int CAS_CTAS = 304, CAS_TH = 256;   // Casimir reduction: CTAs (2 per SM) and threads

int zt_fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int zt_cuda_check(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation)
        return zt_fail(ZT_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return zt_fail(ZT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char* zt_last_error(void) { return g_err; }

// ---- pinned arena of host state mirrors ------------------------------------
#include <mutex>
#include <vector>
namespace {
struct HostChunk {
    zt_dev_state* base;
    int cap;
    std::vector<std::pair<int, int>> free;   // [start, length) ranges, sorted by start
};
std::mutex g_host_mu;
std::vector<HostChunk> g_host_chunks;
constexpr int kHostChunkSlots = 4096;
}  // namespace

zt_dev_state* zt_host_states_acquire(int n) {
    if (n < 1) return nullptr;
    std::lock_guard<std::mutex> g(g_host_mu);
    for (auto& c : g_host_chunks)   // first fit
        for (size_t i = 0; i < c.free.size(); ++i)
            if (c.free[i].second >= n) {
                zt_dev_state* r = c.base + c.free[i].first;
                c.free[i].first += n;
                c.free[i].second -= n;
                if (c.free[i].second == 0) c.free.erase(c.free.begin() + (long)i);
                return r;
            }
    const int cap = n > kHostChunkSlots ? n : kHostChunkSlots;
    void* m = nullptr;
    if (cudaHostAlloc(&m, (size_t)cap * sizeof(zt_dev_state), cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    HostChunk c{(zt_dev_state*)m, cap, {}};
    if (cap > n) c.free.push_back({n, cap - n});
    g_host_chunks.push_back(std::move(c));
    return (zt_dev_state*)m;
}

void zt_host_states_release(zt_dev_state* p, int n) {
    if (!p || n < 1) return;
    std::lock_guard<std::mutex> g(g_host_mu);
    for (auto& c : g_host_chunks) {
        if (p < c.base || p >= c.base + c.cap) continue;
        const int off = (int)(p - c.base);
        size_t i = 0;
        while (i < c.free.size() && c.free[i].first < off) ++i;
        c.free.insert(c.free.begin() + (long)i, {off, n});
        // coalesce with the neighbours
        if (i + 1 < c.free.size() && c.free[i].first + c.free[i].second == c.free[i + 1].first) {
            c.free[i].second += c.free[i + 1].second;
            c.free.erase(c.free.begin() + (long)i + 1);
        }
        if (i > 0 && c.free[i - 1].first + c.free[i - 1].second == c.free[i].first) {
            c.free[i - 1].second += c.free[i].second;
            c.free.erase(c.free.begin() + (long)i);
        }
        return;
    }
}

// Opt-in tracing of host-side phases (environment variable ZT_TRACE=1).
#include <chrono>
static bool trace_on() {
    static int on = -1;
    if (on < 0) {
        const char* e = getenv("ZT_TRACE");
        on = (e && e[0] == '1') ? 1 : 0;
    }
    return on == 1;
}
struct ZtTrace {
    const char* scope;
    std::chrono::steady_clock::time_point t0, last;
    explicit ZtTrace(const char* s) : scope(s) { t0 = last = std::chrono::steady_clock::now(); }
    void mark(const char* what) {
        if (!trace_on()) return;
        auto now = std::chrono::steady_clock::now();
        fprintf(stderr, "[zt-trace] %s %-28s %9.3f ms (total %9.3f ms)\n", scope, what,
                std::chrono::duration<double, std::milli>(now - last).count(),
                std::chrono::duration<double, std::milli>(now - t0).count());
        last = now;
    }
};

#include <mutex>
static std::mutex g_attr_mu;
static unsigned g_attr_done[64];

bool zt_attr_needed(unsigned bit) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return true;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (g_attr_done[dev] & bit) return false;
    g_attr_done[dev] |= bit;
    return true;
}

static int launch_check(zt_plan* p, const char* what) {
    p->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, what);
    return ZT_OK;
}

// ---------------------------------------------------------------------------
// measurement hook
// ---------------------------------------------------------------------------
int zt_timer_begin(zt_plan* p, int kind, double work, double work_alg, cudaStream_t s) {
    if (!p->timing) return -1;
    if (p->nrecs == p->caprecs) {
        const int cap = p->caprecs ? 2 * p->caprecs : 64;
        zt_timer_rec* n = new (std::nothrow) zt_timer_rec[cap];
        if (!n) return -1;
        for (int i = 0; i < p->caprecs; ++i) n[i] = p->recs[i];
        delete[] p->recs;
        p->recs = n;
        p->caprecs = cap;
    }
    zt_timer_rec& r = p->recs[p->nrecs];
    if (!r.a && cudaEventCreate(&r.a) != cudaSuccess) return -1;
    if (!r.b && cudaEventCreate(&r.b) != cudaSuccess) return -1;
    r.kind = kind;
    r.sweep = p->cur_sweep;
    r.work = work;
    r.work_alg = work_alg;
    cudaEventRecord(r.a, s);
    return p->nrecs++;
}

void zt_timer_end(zt_plan* p, int idx, cudaStream_t s) {
    if (idx >= 0) cudaEventRecord(p->recs[idx].b, s);
}

static int timer_collect(zt_plan* p, int iters, int final_tag) {
    for (int i = 0; i < p->nrecs; ++i) {
        zt_timer_rec& r = p->recs[i];
        const bool count = (r.sweep < 0) || (r.sweep < iters) || (r.sweep == final_tag) || iters < 0;
        ZT_CU(cudaEventSynchronize(r.b));
        if (!count) continue;
        float ms = 0.f;
        ZT_CU(cudaEventElapsedTime(&ms, r.a, r.b));
        p->t_n[r.kind]++;
        p->t_ms[r.kind] += ms;
        p->t_work[r.kind] += r.work;
        p->t_work_alg[r.kind] += r.work_alg;
    }
    p->nrecs = 0;
    return ZT_OK;
}

int zt_timer_collect(zt_plan* p, int iters) { return timer_collect(p, iters, -2); }

extern "C" int zt_plan_set_timing(zt_plan* p, int enable) {
    if (!p) return zt_fail(ZT_EINVAL, "plan is NULL");
    int rc = timer_collect(p, -1, -2);
    if (rc) return rc;
    p->timing = enable ? 1 : 0;
    if (p->d_units) ZT_CU(cudaMemset(p->d_units, 0, sizeof(unsigned long long)));
    for (int k = 0; k < ZT_KERNEL_KINDS; ++k) {
        p->t_n[k] = 0;
        p->t_ms[k] = p->t_work[k] = p->t_work_alg[k] = 0.0;
    }
    return ZT_OK;
}

extern "C" int zt_plan_kernel_time(zt_plan* p, int kind, long* launches, double* total_ms, double* work,
                                   double* work_alg) {
    if (!p) return zt_fail(ZT_EINVAL, "plan is NULL");
    if (kind < 0 || kind >= ZT_KERNEL_KINDS) return zt_fail(ZT_EINVAL, "bad kernel kind %d", kind);
    int rc = timer_collect(p, -1, -2);
    if (rc) return rc;
    if (launches) *launches = p->t_n[kind];
    if (total_ms) *total_ms = p->t_ms[kind];
    double extra = 0.0;
    if (kind == ZT_KERNEL_PRODUCT && p->d_units) {   // split products: units issued on the device
        unsigned long long units = 0;
        ZT_CU(cudaDeviceSynchronize());
        ZT_CU(cudaMemcpy(&units, p->d_units, sizeof units, cudaMemcpyDeviceToHost));
        extra = (double)units * 2.0 * 128.0 * 256.0 * 64.0;
    }
    if (work) *work = p->t_work[kind] + extra;
    if (work_alg) *work_alg = p->t_work_alg[kind];
    return ZT_OK;
}

// ---------------------------------------------------------------------------
// Constant per-diagonal data (Sec. 3.2, Eq. 13) and LDL^T factors,
// computed once per plan on the host (the recurrence is sequential along each
// diagonal; on the device it would compete for the FP64 pipe with running
// work).  Entries go to packed lower-triangular arrays at (r, c) = (i + m, i).
// For m = 0 only the leading N-1 equations are factored (the l = 0 mode is
// projected out); the dropped row gets l = 0, -1/d = 0.
// ---------------------------------------------------------------------------
static void factor_diagonal(int N, int m, double* lap_a, double* lap_b, double* fac_l, double* fac_nd) {
    const int n = N - m;
    const int ns = (m == 0) ? N - 1 : n;   // size of the factored system
    const double s = (N - 1) / 2.0;
    double d = 0.0, bprev = 0.0;
    for (int i = 0; i < n; ++i) {
        const double di = (double)i;
        const double a = 2.0 * (s * (2.0 * di + 1.0 + m) - di * (di + m));
        double b = 0.0;
        if (i < n - 1)
            b = -sqrt((di + m + 1.0) * (N - 1.0 - di - m)) * sqrt((di + 1.0) * (N - 1.0 - di));
        const size_t at = zt_tri(i + m, i);
        lap_a[at] = a;
        lap_b[at] = b;
        double l = 0.0, nd = 0.0;
        if (i < ns) {
            if (i == 0) {
                d = a;
            } else {
                l = bprev / d;
                d = a - l * bprev;
            }
            nd = -1.0 / d;
        }
        fac_l[at] = l;
        fac_nd[at] = nd;
        bprev = b;
    }
}

#include <thread>
#include <vector>

static void factor_host(int N, double* lap_a, double* lap_b, double* fac_l, double* fac_nd) {
    unsigned nt = std::thread::hardware_concurrency();
    nt = nt == 0 ? 1 : (nt > 16 ? 16 : nt);
    if ((long long)N * N < 1 << 20) nt = 1;
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([=] {
            for (int m = (int)t; m < N; m += (int)nt) factor_diagonal(N, m, lap_a, lap_b, fac_l, fac_nd);
        });
    for (auto& x : th) x.join();
}

// ---------------------------------------------------------------------------
// W = Delta_N P, elementwise over the matrix: element (r, c) lies on diagonal
// |r - c| at position min(r, c); the block -T_m couples it to its neighbours
// (r-1, c-1) and (r+1, c+1) on the same diagonal.
// ---------------------------------------------------------------------------
__global__ void laplacian_kernel(const double2* __restrict__ P, double2* __restrict__ W,
                                 const double* __restrict__ la, const double* __restrict__ lb, int N) {
    const int r = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int hi = max(r, c), lo = min(r, c);
    const double a = la[zt_tri(hi, lo)];
    const double2 p = P[(size_t)r * N + c];
    double vx = a * p.x, vy = a * p.y;
    if (lo > 0) {
        const double b = lb[zt_tri(hi - 1, lo - 1)];
        const double2 q = P[(size_t)(r - 1) * N + (c - 1)];
        vx = fma(b, q.x, vx);
        vy = fma(b, q.y, vy);
    }
    if (hi < N - 1) {
        const double b = lb[zt_tri(hi, lo)];
        const double2 q = P[(size_t)(r + 1) * N + (c + 1)];
        vx = fma(b, q.x, vx);
        vy = fma(b, q.y, vy);
    }
    W[(size_t)r * N + c] = make_double2(-vx, -vy);
}

int zt_launch_laplacian(zt_plan* p, const double2* P, double2* W, cudaStream_t s) {
    const int N = p->N;
    dim3 grid((N + 127) / 128, N);
    laplacian_kernel<<<grid, 128, 0, s>>>(P, W, p->lap_a, p->lap_b, N);
    return launch_check(p, "laplacian_kernel");
}


// ---------------------------------------------------------------------------
// Fixed-point update (Eq. 9 with the products of Sec. 3.1) and the
// assembly of W_{n+1} (second line of Eq. 8):
//   out = base + h/2 (A - A^H) + c2 B,     c2 = +h^2/4 (sweep), -h^2/4 (final)
// computed on the lower triangle and mirrored (out stays skew-Hermitian; the
// diagonal keeps its imaginary part only).  With `partials`, each CTA also
// writes its share of ||out - old||_F^2.  32x32 tiles over the lower triangle.
// ---------------------------------------------------------------------------
namespace {
constexpr int UT = 32;
}

// Fixed-order reduction of the residual partials and the stop decision.
__device__ __forceinline__ void converge_body(const double* __restrict__ partials, int n, zt_dev_state* st) {
    if (st->done) return;
    __shared__ double sh[256];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += 256) s += __ldcg(partials + k);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double r = sqrt(sh[0]);
        st->iters += 1;
        st->residual = r;
        if (!isfinite(r)) {
            st->nonfinite = 1;
            st->done = 1;
        } else if (r < st->tol) {
            st->converged = 1;
            st->done = 1;
        } else if (st->iters >= st->maxit || st->timeout) {
            st->done = 1;
        }
    }
}

__device__ __forceinline__ void update_body(const UpdateArgs& ua, int t) {
    if (zt_gate_skip(ua.st, ua.gate)) return;
    const double2* __restrict__ base = ua.base;
    const double2* __restrict__ A = ua.A;
    const double2* __restrict__ B = ua.B;
    const double2* old = ua.old;
    double2* out = ua.out;
    const double h2 = ua.h2, c2 = ua.c2;
    double* partials = ua.partials;
    const int N = ua.N;
    __shared__ double2 sAT[UT][UT + 1];
    __shared__ double2 sOut[UT][UT + 1];
    __shared__ double2 sDiag[UT];   // old values on the tile's diagonal
    __shared__ double sred[256];
    int bi = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while (bi * (bi + 1) / 2 > t) --bi;
    while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
    const int bj = t - bi * (bi + 1) / 2;
    const int i0 = bi * UT, j0 = bj * UT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;

    for (int q = 0; q < UT / 8; ++q) {   // sAT[jj][ii] = A[j0+jj, i0+ii]
        const int jj = ty + 8 * q, j = j0 + jj, i = i0 + tx;
        sAT[jj][tx] = (j < N && i < N) ? A[(size_t)j * N + i] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    // ||out - old||_F^2 over the whole matrix = 2 (sum over the lower triangle) - (sum over
    // the diagonal): the per-element weight costs no FP64 instruction (the FP64 pipe is
    // narrow on GB300), the diagonal's share is taken once per diagonal tile below
    double acc = 0.0;
    for (int q = 0; q < UT / 8; ++q) {
        const int ii = ty + 8 * q, jj = tx, i = i0 + ii, j = j0 + jj;
        if (i < N && j < N && i >= j) {
            const size_t e = (size_t)i * N + j;
            const double2 a = A[e], at = sAT[jj][ii], bb = B[e], w = base[e];
            double2 v;
            v.x = w.x + h2 * (a.x - at.x) + c2 * bb.x;
            v.y = w.y + h2 * (a.y + at.y) + c2 * bb.y;
            if (i == j) v.x = 0.0;
            if (partials) {
                const double2 o = old[e];   // read before out[e] is written (old may be out)
                const double dx = v.x - o.x, dy = v.y - o.y;
                acc = fma(dx, dx, fma(dy, dy, acc));
                if (i == j) sDiag[ii] = o;
            }
            out[e] = v;
            sOut[ii][jj] = v;
        }
    }
    __syncthreads();
    if (partials && bi == bj && ty == 0) {   // the tile's diagonal, counted once
        const int i = i0 + tx;
        if (i < N) {
            const double2 v = sOut[tx][tx], o = sDiag[tx];
            const double dx = v.x - o.x, dy = v.y - o.y;
            acc = fma(-0.5 * dx, dx, fma(-0.5 * dy, dy, acc));
        }
    }
    for (int q = 0; q < UT / 8; ++q) {   // mirror: out[j, i] = -conj(out[i, j]), the sign by its bit
        const int jj = ty + 8 * q, ii = tx, i = i0 + ii, j = j0 + jj;
        if (i < N && j < N && i > j) {
            const double2 v = sOut[ii][jj];
            out[(size_t)j * N + i] = make_double2(neg(v.x), v.y);
        }
    }
    if (partials) {
        sred[threadIdx.x] = acc;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) sred[threadIdx.x] += sred[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) partials[t] = 2.0 * sred[0];
    }
    // the launch's last CTA: residual and stop decision (sweeps) or the finalised mark
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        // acq_rel at GPU scope: releases this CTA's partial and stores (ordered before
        // it by the barrier), and the last CTA acquires every other CTA's
        unsigned int prev;
        asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(prev) : "l"(ua.done) : "memory");
        last = prev == (unsigned int)ua.nctas - 1u;
    }
    __syncthreads();
    if (!last) return;
    if (partials) converge_body(partials, ua.nctas, ua.st);
    else if (threadIdx.x == 0 && ua.st->done) {   // W_{n+1} written by every CTA
        ua.st->finalized = 1;
        ua.st->hist = ua.st->converged;   // the next step may extrapolate from this one
    }
    if (threadIdx.x == 0) *ua.done = 0u;
}

__global__ void __launch_bounds__(256) update_kernel(const UpdateArgs a) { update_body(a, blockIdx.x); }

__global__ void __launch_bounds__(256) update_grouped(const UpdateArgs* tab, const int* offs, int n, int gate) {
    const int inst = zt_group_find(offs, n, blockIdx.x);
    UpdateArgs a = tab[inst];
    a.gate = gate;
    update_body(a, blockIdx.x - offs[inst]);
}

int zt_update_ctas(int N) {
    const int nt = (N + UT - 1) / UT;
    return nt * (nt + 1) / 2;
}

int zt_update_grouped(const UpdateArgs* tab, const int* offs, int n, int total, cudaStream_t s, int gate) {
    update_grouped<<<total, 256, 0, s>>>(tab, offs, n, gate);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "update_grouped");
    return ZT_OK;
}

// keep_hist = 0 drops the history (another W or h than the plan's previous step).
__global__ void state_init_kernel(zt_dev_state* st, double tol, int maxit, int keep_hist) {
    if (!keep_hist) st->hist = 0;
    st->done = 0;
    st->iters = 0;
    st->converged = 0;
    st->nonfinite = 0;
    st->timeout = 0;
    st->maxit = maxit;
    st->residual = 0.0;
    st->tol = tol;
    st->finalized = 0;
}

// Start of a step: the first iterate Wt^0 (the extrapolated midpoint when the
// plan's history allows it, else W_n) and the copy of W_n kept for the next
// step's extrapolation.  Runs after state_init_kernel on the same stream.
__global__ void __launch_bounds__(256) step_start_kernel(const double2* __restrict__ W, double2* __restrict__ Wn,
                                                         double2* __restrict__ Wt, long long count,
                                                         const zt_dev_state* __restrict__ st) {
    const int hist = st->hist;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const double2 w = W[i];
        Wt[i] = hist ? zt_extrapolate(w, Wn[i]) : w;
        Wn[i] = w;
    }
}

static int launch_update(zt_plan* p, const double2* base, const double2* old, double2* out,
                         double h, double sign_b, bool resid, cudaStream_t s, int gate) {
    const int N = p->N;
    const int nt = (N + UT - 1) / UT;
    const int ntiles = nt * (nt + 1) / 2;
    // lower triangle: base, A, A^T, B (+ old) read, out written twice
    const double tri = 16.0 * N * (N + 1.0) / 2.0;
    const double bytes = tri * ((resid ? 5.0 : 4.0) + 2.0);
    UpdateArgs ua;
    ua.base = base;
    ua.A = p->A;
    ua.B = p->B;
    ua.old = old;
    ua.out = out;
    ua.h2 = h / 2.0;
    ua.c2 = sign_b * h * h / 4.0;
    ua.partials = resid ? p->partials : nullptr;
    ua.N = N;
    ua.final_write = resid ? 0 : 1;
    ua.st = p->state;
    ua.gate = gate;
    ua.done = p->upd_done;   // the last CTA: residual and stop decision, or the finalised mark
    ua.nctas = ntiles;
    const int t = zt_timer_begin(p, ZT_KERNEL_UPDATE, bytes, bytes, s);
    update_kernel<<<ntiles, 256, 0, s>>>(ua);
    zt_timer_end(p, t, s);
    return launch_check(p, "update_kernel");
}

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
static int zgemm(zt_plan* p, const double2* X, const double2* Y, double2* C, double alpha,
                 int lower_only, cudaStream_t s, int gate) {
    if (p->precision == ZT_PRECISION_SPLIT)
        return zt_launch_zgemm_split(p, X, Y, C, alpha, lower_only, s, gate);
    return zt_launch_zgemm_fp64(p, X, Y, C, alpha, lower_only, s, gate);
}

extern "C" void zt_plan_destroy(zt_plan* p) {
    if (!p) return;
    cudaStream_t ms = p->mstream;
    if (!ms) {   // creation failed before the private stream existed: nothing was allocated
        zt_host_states_release(p->h_state, 1);
        delete p;
        return;
    }
    if (p->last_use) cudaStreamWaitEvent(ms, p->last_use, 0);   // frees after the plan's last work
    if (p->split) zt_split_destroy(p);
    zt_solve_destroy(p);
    zt_dfree(p->lap_a, ms);
    zt_dfree(p->lap_b, ms);
    zt_dfree(p->Wn, ms);
    zt_dfree(p->Wt, ms);
    zt_dfree(p->P, ms);
    zt_dfree(p->A, ms);
    zt_dfree(p->B, ms);
    zt_dfree(p->partials, ms);
    zt_dfree(p->cas_part, ms);
    zt_dfree(p->state, ms);
    zt_dfree(p->upd_done, ms);
    zt_dfree(p->d_units, ms);
    zt_host_states_release(p->h_state, 1);   // no copy into it is in flight: steps end synchronised
    for (int i = 0; i < p->caprecs; ++i) {
        if (p->recs[i].a) cudaEventDestroy(p->recs[i].a);
        if (p->recs[i].b) cudaEventDestroy(p->recs[i].b);
    }
    delete[] p->recs;
    if (p->last_use) cudaEventDestroy(p->last_use);
    cudaStreamDestroy(ms);   // returns at once; the frees complete in stream order
    delete p;
}

static void fill_tuning_defaults(zt_tuning& t) {
    if (t.slices == 0) t.slices = 7;
    if (t.digit_bits == 0) t.digit_bits = 7;
    if (t.exact_groups == 0) t.exact_groups = 4;
    if (t.wait_us == 0) t.wait_us = 2000000;
}

extern "C" long long zt_plan_estimate_bytes(int N, int precision, const zt_tuning* opt) {
    if (N < 1 || N > 16384) return -1;
    zt_tuning t{};
    if (opt) t = *opt;
    fill_tuning_defaults(t);
    const size_t nn = (size_t)N * N, ntri = (size_t)N * (N + 1) / 2;
    const size_t nt = (N + 31) / 32;
    size_t b = 2 * ntri * 8 + 5 * nn * 16 + nt * (nt + 1) / 2 * 8 + zt_solve_bytes(N) + 1024 +
               ((size_t)CAS_CTAS + 1) * 8 * sizeof(double);
    if (precision == ZT_PRECISION_SPLIT) b += zt_split_bytes(N, t);
    return (long long)b;
}

extern "C" int zt_plan_create(int N, int precision, const zt_tuning* opt, zt_plan** out) {
    if (!out) return zt_fail(ZT_EINVAL, "zt_plan_create: out is NULL");
    *out = nullptr;
    if (N < 1 || N > 16384) return zt_fail(ZT_EINVAL, "zt_plan_create: N=%d outside [1, 16384]", N);
    if (precision != ZT_PRECISION_FP64 && precision != ZT_PRECISION_SPLIT)
        return zt_fail(ZT_EINVAL, "zt_plan_create: unknown precision %d", precision);
    zt_plan* p = new (std::nothrow) zt_plan();
    if (!p) return zt_fail(ZT_ENOMEM, "zt_plan_create: host allocation failed");
    p->N = N;
    p->precision = precision;
    if (opt) p->tun = *opt;
    fill_tuning_defaults(p->tun);
    if (p->tun.final_mode != ZT_FINAL_FRESH && p->tun.final_mode != ZT_FINAL_REUSE) {
        delete p;
        return zt_fail(ZT_EINVAL, "zt_plan_create: bad final_mode %d", opt->final_mode);
    }
    if (p->tun.sweeps_per_sync < 0 || p->tun.sweeps_per_sync > 64) {
        delete p;
        return zt_fail(ZT_EINVAL, "zt_plan_create: sweeps_per_sync outside [0, 64]");
    }
    if (p->tun.first_iterate != ZT_FIRST_EXTRAPOLATED && p->tun.first_iterate != ZT_FIRST_WN) {
        delete p;
        return zt_fail(ZT_EINVAL, "zt_plan_create: bad first_iterate %d", p->tun.first_iterate);
    }
    if (precision == ZT_PRECISION_SPLIT) {   // checked before any device work
        const zt_tuning& t = p->tun;
        const char* bad = nullptr;
        if (t.slices < 3 || t.slices > 8) bad = "slices outside [3, 8]";
        else if (t.digit_bits < 6 || t.digit_bits > 8) bad = "digit_bits outside [6, 8]";
        else if (t.exact_groups < 1 || t.exact_groups > t.slices) bad = "exact_groups outside [1, slices]";
        else if (t.slices * t.digit_bits > 62) bad = "slices*digit_bits above 62";
        else if (t.tile_order < 0 || t.tile_order > 6) bad = "tile_order outside [0, 6]";
        else if (t.no_persistent != 0 && t.no_persistent != 1) bad = "no_persistent must be 0 or 1";
        else if (t.wait_us < 1 || t.wait_us > 60000000) bad = "wait_us outside [1, 60000000]";
        else if (t.debug_stall_loads < 0) bad = "debug_stall_loads must be >= 0";
        else if (t.slices2 != 0 && (t.slices2 < 2 || t.slices2 > t.slices)) bad = "slices2 outside [2, slices]";
        else if (t.second_form < 0 || t.second_form > 2) bad = "second_form outside [0, 2]";
        if (bad) {
            delete p;
            return zt_fail(ZT_EINVAL, "zt_plan_create: %s", bad);
        }
    }
    int rc = ZT_OK;
    auto fail = [&](int code) {
        zt_plan_destroy(p);
        return code;
    };
#define ZT_TRY(call)                                         \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return fail(zt_cuda_check(_e, #call)); \
    } while (0)
    ZtTrace tr("zt_plan_create");
    ZT_TRY(cudaGetDevice(&p->device));
    if (zt_attr_needed(ZT_ATTR_POOL)) {
        // Plans allocate from the device's stream-ordered pool.  With the default
        // release threshold (0) memory freed by a destroyed plan is handed back to
        // the system at later synchronisations, which can stall unrelated steps;
        // keeping it in the pool makes the next plan's allocation a reuse.
        cudaMemPool_t pool = nullptr;
        if (cudaDeviceGetDefaultMemPool(&pool, p->device) == cudaSuccess) {
            cuuint64_t keep = ~(cuuint64_t)0;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    ZT_TRY(zt_setup_stream(&p->mstream));
    tr.mark("stream");
    ZT_TRY(cudaEventCreateWithFlags(&p->last_use, cudaEventDisableTiming));
    cudaStream_t cs = p->mstream;
    const size_t ntri = (size_t)N * (N + 1) / 2;
    const size_t mat = (size_t)N * N * sizeof(double2);
    ZT_TRY(ZT_DMALLOC(p->lap_a, ntri * sizeof(double), cs));
    ZT_TRY(ZT_DMALLOC(p->lap_b, ntri * sizeof(double), cs));
    ZT_TRY(ZT_DMALLOC(p->Wn, mat, cs));
    ZT_TRY(ZT_DMALLOC(p->Wt, mat, cs));
    ZT_TRY(ZT_DMALLOC(p->P, mat, cs));
    ZT_TRY(ZT_DMALLOC(p->A, mat, cs));
    ZT_TRY(ZT_DMALLOC(p->B, mat, cs));
    const int nt = (N + UT - 1) / UT;
    p->npartials = nt * (nt + 1) / 2;
    ZT_TRY(ZT_DMALLOC(p->partials, (size_t)p->npartials * sizeof(double), cs));
    ZT_TRY(ZT_DMALLOC(p->cas_part, ((size_t)CAS_CTAS + 1) * 8 * sizeof(double), cs));
    ZT_TRY(ZT_DMALLOC(p->state, sizeof(zt_dev_state), cs));
    ZT_TRY(ZT_DMALLOC(p->upd_done, 16, cs));
    ZT_TRY(cudaMemsetAsync(p->upd_done, 0, 16, cs));
    ZT_TRY(ZT_DMALLOC(p->d_units, sizeof(unsigned long long), cs));
    tr.mark("allocations");
    p->h_state = zt_host_states_acquire(1);
    if (!p->h_state) return fail(zt_fail(ZT_ENOMEM, "pinned host allocation failed"));
    // set-up work runs on a private stream so that creating a plan does not
    // wait for work other threads have queued on the device
    rc = zt_solve_create(p);
    if (rc != ZT_OK) return fail(rc);
    tr.mark("solve workspace");
    cudaMemsetAsync(p->state, 0, sizeof(zt_dev_state), cs);
    cudaMemsetAsync(p->d_units, 0, sizeof(unsigned long long), cs);
    {
        std::vector<double> ha, hb, hl, hn;
        try {
            ha.resize(ntri);
            hb.resize(ntri);
            hl.resize(ntri);
            hn.resize(ntri);
        } catch (...) {
            return fail(zt_fail(ZT_ENOMEM, "host allocation for the Laplacian factors failed"));
        }
        tr.mark("host vectors");
        factor_host(N, ha.data(), hb.data(), hl.data(), hn.data());
        tr.mark("host factors");
        cudaMemcpyAsync(p->lap_a, ha.data(), ntri * sizeof(double), cudaMemcpyHostToDevice, cs);
        cudaMemcpyAsync(p->lap_b, hb.data(), ntri * sizeof(double), cudaMemcpyHostToDevice, cs);
        cudaError_t se = cudaGetLastError();
        if (se == cudaSuccess) se = cudaStreamSynchronize(cs);   // host vectors go out of scope
        if (se != cudaSuccess) return fail(zt_cuda_check(se, "plan set-up (factor upload)"));
        tr.mark("factor upload + sync");
        rc = zt_solve_upload_factors(p, hl.data(), hn.data());
        if (rc != ZT_OK) return fail(rc);
        tr.mark("solve factors");
    }
    if (precision == ZT_PRECISION_SPLIT) {
        rc = zt_split_create(p);
        if (rc != ZT_OK) return fail(rc);
    }
    tr.mark("split workspace");
    ZT_TRY(cudaStreamSynchronize(cs));   // allocations and set-up visible to every stream
    tr.mark("final sync");
#undef ZT_TRY
    *out = p;
    return ZT_OK;
}

extern "C" long zt_plan_launch_count(const zt_plan* p) { return p ? p->launches : 0; }

extern "C" void zt_plan_reset_history(zt_plan* p) {
    if (p) p->last_W = nullptr;   // the next step's state_init drops the device history too
}

static int check_ptr(const void* ptr, const char* name) {
    if (!ptr) return zt_fail(ZT_EINVAL, "%s is NULL", name);
    if (((uintptr_t)ptr & 15u) != 0) return zt_fail(ZT_EINVAL, "%s is not 16-byte aligned", name);
    return ZT_OK;
}

// ---------------------------------------------------------------------------
// public entry points
// ---------------------------------------------------------------------------
extern "C" int zeitlin_laplacian_apply(zt_plan* p, const double* P, double* W, void* stream) {
    if (!p) return zt_fail(ZT_EINVAL, "plan is NULL");
    int rc;
    if ((rc = check_ptr(P, "P")) || (rc = check_ptr(W, "W"))) return rc;
    if (P == W) return zt_fail(ZT_EINVAL, "W must not alias P");
    rc = zt_launch_laplacian(p, (const double2*)P, (double2*)W, (cudaStream_t)stream);
    zt_note_use(p, (cudaStream_t)stream);
    return rc;
}

extern "C" int zeitlin_stream_solve(zt_plan* p, const double* W, double* P, void* stream) {
    if (!p) return zt_fail(ZT_EINVAL, "plan is NULL");
    int rc;
    if ((rc = check_ptr(P, "P")) || (rc = check_ptr(W, "W"))) return rc;
    if (P == W) return zt_fail(ZT_EINVAL, "P must not alias W");
    rc = zt_launch_stream_solve(p, (const double2*)W, (double2*)P, (cudaStream_t)stream, ZT_GATE_NONE);
    zt_note_use(p, (cudaStream_t)stream);
    return rc;
}

extern "C" int zt_zgemm_skew(zt_plan* p, const double* X, const double* Y, double* C, void* stream) {
    if (!p) return zt_fail(ZT_EINVAL, "plan is NULL");
    int rc;
    if ((rc = check_ptr(X, "X")) || (rc = check_ptr(Y, "Y")) || (rc = check_ptr(C, "C"))) return rc;
    if (C == X || C == Y) return zt_fail(ZT_EINVAL, "C must not alias X or Y");
    cudaStream_t s = (cudaStream_t)stream;
    if (p->precision == ZT_PRECISION_SPLIT) {
        ZT_CU(cudaMemsetAsync(p->state, 0, sizeof(zt_dev_state), s));
        rc = zgemm(p, (const double2*)X, (const double2*)Y, (double2*)C, -1.0, 0, s, ZT_GATE_NONE);
        if (rc) return rc;
        ZT_CU(cudaMemcpyAsync(p->h_state, p->state, sizeof(zt_dev_state), cudaMemcpyDeviceToHost, s));
        ZT_CU(cudaStreamSynchronize(s));
        if (p->h_state->timeout) return zt_fail(ZT_ETIMEOUT, "zt_zgemm_skew: bounded device wait ran out");
        return ZT_OK;
    }
    rc = zgemm(p, (const double2*)X, (const double2*)Y, (double2*)C, -1.0, 0, s, ZT_GATE_NONE);
    zt_note_use(p, s);
    return rc;
}

// ---------------------------------------------------------------------------
// Casimirs C_k = tr(W^k), k = 2..5 (Sec. 2, Eq. 7), from W^2 = W W and
// W^4 = W^2 W^2 (the plan's products) and conjugate dot products: W is
// skew-Hermitian and W^2, W^4 are Hermitian, so tr(X Y) = sum_ij X_ij Y_ji
// = -sum_ij X_ij conj(W_ij) for Y = W and +sum_ij X_ij conj(Y_ij) for Y = W^2:
//   C2 = -sum |W_ij|^2,  C3 = -sum (W^2)_ij conj(W_ij),
//   C4 = sum |(W^2)_ij|^2,  C5 = -sum (W^4)_ij conj(W_ij).
// FP64 sums in a fixed order (per-CTA partials, then one pass).
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(CAS_TH) casimir_partials(const double2* __restrict__ W,
                                                           const double2* __restrict__ W2,
                                                           const double2* __restrict__ W4, size_t n,
                                                           double* __restrict__ part) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (size_t e = (size_t)blockIdx.x * CAS_TH + threadIdx.x; e < n; e += (size_t)gridDim.x * CAS_TH) {
        const double2 w = W[e], a = W2[e], b = W4[e];
        acc[0] -= w.x * w.x + w.y * w.y;
        acc[2] -= a.x * w.x + a.y * w.y;
        acc[3] -= a.y * w.x - a.x * w.y;
        acc[4] += a.x * a.x + a.y * a.y;
        acc[6] -= b.x * w.x + b.y * w.y;
        acc[7] -= b.y * w.x - b.x * w.y;
    }
    __shared__ double red[CAS_TH];
    for (int j = 0; j < 8; ++j) {
        red[threadIdx.x] = acc[j];
        __syncthreads();
        for (int w = CAS_TH / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(size_t)blockIdx.x * 8 + j] = red[0];
        __syncthreads();
    }
}

__global__ void casimir_final(const double* __restrict__ part, int nparts, double* __restrict__ out) {
    const int j = threadIdx.x;
    if (j >= 8) return;
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += part[(size_t)b * 8 + j];
    out[j] = s;
}

extern "C" int zeitlin_casimirs(zt_plan* p, const double* W, double* C, void* stream) {
    if (!p) return zt_fail(ZT_EINVAL, "plan is NULL");
    if (!C) return zt_fail(ZT_EINVAL, "C is NULL");
    int rc;
    if ((rc = check_ptr(W, "W"))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    ZT_CU(cudaMemsetAsync(p->state, 0, sizeof(zt_dev_state), s));
    if ((rc = zgemm(p, (const double2*)W, (const double2*)W, p->A, -1.0, 0, s, ZT_GATE_NONE))) return rc;   // W W
    if ((rc = zgemm(p, p->A, p->A, p->B, 1.0, 0, s, ZT_GATE_NONE))) return rc;   // W^2 W^2 (W^2 Hermitian)
    const size_t n = (size_t)p->N * p->N;
    casimir_partials<<<CAS_CTAS, CAS_TH, 0, s>>>((const double2*)W, p->A, p->B, n, p->cas_part);
    casimir_final<<<1, 32, 0, s>>>(p->cas_part, CAS_CTAS, p->cas_part + (size_t)CAS_CTAS * 8);
    p->launches += 2;
    ZT_CU(cudaGetLastError());
    ZT_CU(cudaMemcpyAsync(p->h_state, p->state, sizeof(zt_dev_state), cudaMemcpyDeviceToHost, s));
    ZT_CU(cudaMemcpyAsync(C, p->cas_part + (size_t)CAS_CTAS * 8, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    ZT_CU(cudaStreamSynchronize(s));
    zt_note_use(p, s);
    if (p->h_state->timeout) return zt_fail(ZT_ETIMEOUT, "zeitlin_casimirs: bounded device wait ran out");
    return ZT_OK;
}

// One fixed-point sweep (Eq. 9): Pt = solve(Wt), A = Pt Wt,
// B = A Pt, Wt <- W_n + h/2 (A - A^H) + h^2/4 B, residual, stop decision.
// Pt = solve(Wk), A = Pt Wk, B = A Pt (lower half), Wk the current iterate.
static int enqueue_products(zt_plan* p, const double2* Wk, cudaStream_t s, int gate) {
    int rc;
    if ((rc = zt_launch_stream_solve(p, Wk, p->P, s, gate))) return rc;
    if (p->precision == ZT_PRECISION_SPLIT) {
        // The product kernel forms X conj(Y)^T from the X' planes (rows of X) and a
        // B'^T slot (rows of Y).  A = Pt Wt = -Pt conj(Wt)^T (Wt skew-Hermitian), and
        // B = A Pt = Pt Wt Pt is skew-Hermitian, so B = -B^H = -Pt^H A^H = Pt A^H = Pt conj(A)^T:
        // both products take Pt's X' planes, split once.  Pt into the X' planes and Wt
        // into slot 0 in one launch, then A into slot 1.
        if ((rc = zt_split_operands2(p, p->P, Wk, s, gate))) return rc;
        if ((rc = zt_split_product(p, 0, p->A, -1.0, 0, 1, s, gate))) return rc;   // A = Pt Wt
        if ((rc = zt_split_operand(p, p->A, 0, 1, s, gate))) return rc;            // A: B'^T slot 1
        return zt_split_product(p, 1, p->B, +1.0, 1, 0, s, gate);                   // B = Pt A^H
    }
    if ((rc = zgemm(p, p->P, Wk, p->A, -1.0, 0, s, gate))) return rc;
    return zgemm(p, p->A, p->P, p->B, -1.0, 1, s, gate);
}

// Sweep k of the step from W = W_n.  W stays W_n until the final assembly
// writes W_{n+1} into it, so it serves as W_n throughout.  The first iterate is
// Wt (written by step_start_kernel) or, without extrapolation, W itself; later
// sweeps read the workspace Wt that every sweep writes.
static int enqueue_sweep(zt_plan* p, int k, const double2* W, bool from_wt, double h, cudaStream_t s) {
    int rc;
    p->cur_sweep = k;
    const double2* Wk = (k == 0 && !from_wt) ? W : p->Wt;
    if ((rc = enqueue_products(p, Wk, s, ZT_GATE_SWEEP))) return rc;
    // the update's last CTA reduces the residual and takes the stop decision
    rc = launch_update(p, W, Wk, p->Wt, h, +1.0, true, s, ZT_GATE_SWEEP);
    p->cur_sweep = -1;
    return rc;
}

// Second line of Eq. 8; runs only once the sweeps are done.
static int enqueue_final(zt_plan* p, int tag, double2* W, double h, cudaStream_t s) {
    int rc;
    p->cur_sweep = tag;
    if (p->tun.final_mode == ZT_FINAL_FRESH && (rc = enqueue_products(p, p->Wt, s, ZT_GATE_FINAL))) return rc;
    // the assembly's last CTA marks the state finalised (W_{n+1} written by every CTA)
    rc = launch_update(p, p->Wt, nullptr, W, h, -1.0, false, s, ZT_GATE_FINAL);
    p->cur_sweep = -1;
    return rc;
}

static int step_impl_(zt_plan* p, double2* W, double h, double tol, int maxit, zt_step_stats* stats,
                      cudaStream_t s);
static int step_impl(zt_plan* p, double2* W, double h, double tol, int maxit, zt_step_stats* stats,
                     cudaStream_t s) {
    const int rc = step_impl_(p, W, h, tol, maxit, stats, s);
    zt_note_use(p, s);
    return rc;
}
static int step_impl_(zt_plan* p, double2* W, double h, double tol, int maxit, zt_step_stats* stats,
                      cudaStream_t s) {
    // first iterate: extrapolated from this plan's previous step when that step
    // advanced the same W with the same h (decided on the device from its history)
    const bool extrap = p->tun.first_iterate == ZT_FIRST_EXTRAPOLATED;
    const int keep = extrap && p->last_W == (const void*)W && p->last_h == h;
    p->last_W = W;
    p->last_h = h;
    state_init_kernel<<<1, 1, 0, s>>>(p->state, tol, maxit, keep);
    int rc = launch_check(p, "state_init_kernel");
    if (rc) return rc;
    if (extrap) {
        const long long nn = (long long)p->N * p->N;
        const int grid = (int)std::min<long long>((nn + 255) / 256, 4096);
        step_start_kernel<<<grid, 256, 0, s>>>(W, p->Wn, p->Wt, nn, p->state);
        if ((rc = launch_check(p, "step_start_kernel"))) return rc;
    }
    int enq = 0, round = 0;
    // sweeps per host check: fixed, or as many as the previous step took (the
    // device gates sweeps past convergence, so a larger chunk only costs launches)
    const int chunk = p->tun.sweeps_per_sync ? p->tun.sweeps_per_sync : (p->last_iters > 0 ? p->last_iters : 4);
    for (;; ++round) {
        for (int c = 0; c < chunk && enq < maxit; ++c, ++enq)
            if ((rc = enqueue_sweep(p, enq, W, extrap, h, s))) return rc;
        if ((rc = enqueue_final(p, ZT_SWEEP_FINAL + round, W, h, s))) return rc;
        ZT_CU(cudaMemcpyAsync(p->h_state, p->state, sizeof(zt_dev_state), cudaMemcpyDeviceToHost, s));
        ZT_CU(cudaStreamSynchronize(s));
        if (p->h_state->done) break;
        if (enq >= maxit) return zt_fail(ZT_ECUDA, "isomp_step: state not done after maxit sweeps");
    }
    const zt_dev_state& hs = *p->h_state;
    if (hs.iters > 0 && !hs.timeout && !hs.nonfinite) p->last_iters = hs.iters;
    if (p->timing && (rc = timer_collect(p, hs.iters, ZT_SWEEP_FINAL + round))) return rc;
    if (stats) {
        stats->iters = hs.iters;
        stats->converged = hs.converged;
        stats->residual = hs.residual;
    }
    if (hs.timeout) return zt_fail(ZT_ETIMEOUT, "isomp_step: a bounded device wait ran out");
    if (hs.nonfinite) return zt_fail(ZT_ENONFINITE, "isomp_step: residual is not finite");
    if (!hs.converged)
        return zt_fail(ZT_NOT_CONVERGED, "isomp_step: no convergence in %d sweeps (residual %.3e)",
                       hs.iters, hs.residual);
    return ZT_OK;
}

static int check_step_args(zt_plan* p, const double* W, double h, double tol, int maxit) {
    if (!p) return zt_fail(ZT_EINVAL, "plan is NULL");
    int rc;
    if ((rc = check_ptr(W, "W"))) return rc;
    if (!std::isfinite(h)) return zt_fail(ZT_EINVAL, "h is not finite");
    if (!(tol >= 0.0)) return zt_fail(ZT_EINVAL, "tol must be >= 0");
    if (maxit < 1 || maxit > 100000) return zt_fail(ZT_EINVAL, "maxit outside [1, 100000]");
    return ZT_OK;
}

extern "C" int isomp_step(zt_plan* p, double* W, double h, double tol, int maxit, zt_step_stats* stats,
                          void* stream) {
    int rc = check_step_args(p, W, h, tol, maxit);
    if (rc) return rc;
    return step_impl(p, (double2*)W, h, tol, maxit, stats, (cudaStream_t)stream);
}

extern "C" int isomp_run(zt_plan* p, double* W, double h, long nsteps, double tol, int maxit,
                         zt_run_stats* stats, void* stream) {
    int rc = check_step_args(p, W, h, tol, maxit);
    if (rc) return rc;
    if (nsteps < 0) return zt_fail(ZT_EINVAL, "nsteps < 0");
    zt_run_stats tot{};
    tot.all_converged = 1;
    int worst = ZT_OK;
    for (long n = 0; n < nsteps; ++n) {
        zt_step_stats st{};
        rc = step_impl(p, (double2*)W, h, tol, maxit, &st, (cudaStream_t)stream);
        if (rc < 0) {
            if (stats) *stats = tot;
            return rc;
        }
        if (rc == ZT_NOT_CONVERGED) worst = ZT_NOT_CONVERGED;
        tot.steps++;
        tot.total_iters += st.iters;
        if (st.iters > tot.max_iters) tot.max_iters = st.iters;
        if (!st.converged) tot.all_converged = 0;
        if (st.residual > tot.max_residual) tot.max_residual = st.residual;
    }
    if (stats) *stats = tot;
    if (worst) return zt_fail(worst, "isomp_run: some steps did not converge");
    return ZT_OK;
}
