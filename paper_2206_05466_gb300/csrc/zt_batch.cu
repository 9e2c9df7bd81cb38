// Grouped IsoMP steps over many independent instances (ensembles, serving).
//
// A batch binds existing plans (each with its own N, precision and
// workspace), their state matrices W and their time steps h.  One batched
// step runs the same sequence as isomp_step, but every kernel is one grouped
// launch over all instances (per-instance arguments in device tables, CTAs
// mapped to instances through prefix sums).  Each instance keeps its own
// device convergence state, so members that converge early are masked off by
// the kernels' gates while the others keep sweeping; one host
// synchronisation per step reads all states.  Optionally the launch sequence
// of a step is captured once into CUDA graphs and replayed.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "zt_internal.h"

namespace {

struct CopyArgs {   // W -> W_n and the first iterate -> Wt, and the instance's step state reset
    const double2* src;
    double2* d1;
    double2* d2;
    long long count;
    zt_dev_state* st;
    int extrap;         // the plan starts from the extrapolated midpoint when its history allows
};
constexpr int COPY_PER_CTA = 256 * 4;

struct Op {          // one grouped launch: table and CTA prefix sums in device memory
    void* tab = nullptr;
    int* offs = nullptr;
    int n = 0;
    int total = 0;
};

}  // namespace

__global__ void __launch_bounds__(256) copy_grouped(const CopyArgs* tab, const int* offs, int n, double tol,
                                                    int maxit) {
    const int inst = zt_group_find(offs, n, blockIdx.x);
    const CopyArgs a = tab[inst];
    // the history flag is read by every CTA and changed only at the end of a step
    const int hist = a.extrap && a.st->hist;
    if (blockIdx.x == offs[inst] && threadIdx.x == 0) {   // the instance's first CTA resets its state
        zt_dev_state* st = a.st;
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
    const long long base = (long long)(blockIdx.x - offs[inst]) * COPY_PER_CTA;
    for (int q = 0; q < 4; ++q) {
        const long long i = base + threadIdx.x + 256 * q;
        if (i < a.count) {   // the same arithmetic as step_start_kernel of a single plan
            const double2 v = a.src[i];
            a.d2[i] = hist ? zt_extrapolate(v, a.d1[i]) : v;
            a.d1[i] = v;
        }
    }
}

__global__ void state_gather(zt_dev_state* const* sts, int n, zt_dev_state* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = *sts[i];
}

struct zt_batch {
    int n = 0;
    int device = 0;
    int final_mode = ZT_FINAL_FRESH;
    int maxN = 0;                    // largest instance
    std::vector<zt_plan*> plans;
    std::vector<double2*> W;
    std::vector<double> h;
    unsigned char* dbuf = nullptr;   // all tables
    cudaStream_t mstream = nullptr;  // private stream of the stream-ordered allocations (no device syncs)
    zt_dev_state** dstates = nullptr;
    zt_dev_state* gathered = nullptr;
    zt_dev_state* hstates = nullptr;   // pinned host copy of the states (also the captured memcpy target)
    Op copy, solve, split_PW, split_A, gemm1, gemm2, f64a, f64b, upd_sweep, upd_final;
    int sweeps_per_sync = 0;    // fixed chunk of sweeps per host check; 0: adaptive
    int last_max = 0;           // largest sweep count of an instance in the previous step
    int g_spc = 0;              // chunk the graphs were captured for
    long launches = 0;
    int use_graph = 0;
    cudaGraphExec_t g_first = nullptr, g_more = nullptr;
    long g_first_k = 0, g_more_k = 0;   // kernels in each graph
    cudaStream_t g_stream = nullptr;   // stream the graphs were captured for (the caller's)
    cudaStream_t own = nullptr;        // non-blocking stream the graphs are captured on and replayed on
    cudaEvent_t ev_in = nullptr;
    int g_tol_maxit_set = 0;
    double g_tol = 0.0;
    int g_maxit = 0;
};

namespace {

// Host-side builder: collects tables, then uploads them in one allocation.
struct Builder {
    std::vector<unsigned char> bytes;
    struct Pending {
        Op* op;
        size_t tab_off, offs_off;
    };
    std::vector<Pending> pend;

    size_t put(const void* src, size_t n, size_t align) {
        size_t off = (bytes.size() + align - 1) / align * align;
        bytes.resize(off + n);
        if (n) std::memcpy(bytes.data() + off, src, n);
        return off;
    }
    template <class T>
    void add(Op* op, const std::vector<T>& tab, const std::vector<int>& ctas) {
        std::vector<int> offs(ctas.size() + 1, 0);
        for (size_t i = 0; i < ctas.size(); ++i) offs[i + 1] = offs[i] + ctas[i];
        op->n = (int)tab.size();
        op->total = offs.back();
        const size_t t = put(tab.data(), tab.size() * sizeof(T), 128);
        const size_t o = put(offs.data(), offs.size() * sizeof(int), 16);
        pend.push_back({op, t, o});
    }
    int upload(zt_batch* b) {
        if (bytes.empty()) return ZT_OK;
        ZT_CU(ZT_DMALLOC(b->dbuf, bytes.size(), b->mstream));
        ZT_CU(cudaMemcpyAsync(b->dbuf, bytes.data(), bytes.size(), cudaMemcpyHostToDevice, b->mstream));
        ZT_CU(cudaStreamSynchronize(b->mstream));   // host staging goes out of scope
        for (auto& q : pend) {
            q.op->tab = b->dbuf + q.tab_off;
            q.op->offs = reinterpret_cast<int*>(b->dbuf + q.offs_off);
        }
        return ZT_OK;
    }
};

int count_launch(zt_batch* b, const char* what) {
    b->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, what);
    return ZT_OK;
}

// Pt = solve(Wt), A = Pt Wt, B = A Pt (in split form as Pt A^H) for every instance
// (grouped launches).
int enqueue_products(zt_batch* b, cudaStream_t s, int gate) {
    int rc;
    if ((rc = zt_solve_grouped((const SolveArgs*)b->solve.tab, b->solve.offs, b->solve.n, b->solve.total, b->maxN,
                               s, gate)))
        return rc;
    b->launches += ZT_SOLVE_LAUNCHES;
    if (b->gemm1.n) {
        // Pt into the X' planes, Wt into B'^T slot 0: one launch; then A into slot 1 and
        // B = Pt A^H (the same form as the single-plan path)
        if ((rc = zt_split_rows_grouped((const SplitRowsArgs*)b->split_PW.tab, b->split_PW.offs, b->split_PW.n,
                                        b->split_PW.total, s, gate)))
            return rc;
        if ((rc = zt_split_gemm_grouped((const GemmEntry*)b->gemm1.tab, b->gemm1.offs, b->gemm1.n, b->gemm1.total,
                                        s, gate)))
            return rc;
        if ((rc = zt_split_rows_grouped((const SplitRowsArgs*)b->split_A.tab, b->split_A.offs, b->split_A.n,
                                        b->split_A.total, s, gate)))
            return rc;
        if ((rc = zt_split_gemm_grouped((const GemmEntry*)b->gemm2.tab, b->gemm2.offs, b->gemm2.n, b->gemm2.total,
                                        s, gate)))
            return rc;
        b->launches += 4;
    }
    if (b->f64a.n) {
        if ((rc = zt_fp64_gemm_grouped((const Fp64GemmArgs*)b->f64a.tab, b->f64a.offs, b->f64a.n, b->f64a.total, s,
                                       gate)))
            return rc;
        if ((rc = zt_fp64_gemm_grouped((const Fp64GemmArgs*)b->f64b.tab, b->f64b.offs, b->f64b.n, b->f64b.total, s,
                                       gate)))
            return rc;
        b->launches += 2;
    }
    return ZT_OK;
}

int enqueue_sweep(zt_batch* b, cudaStream_t s) {
    int rc;
    if ((rc = enqueue_products(b, s, ZT_GATE_SWEEP))) return rc;
    if ((rc = zt_update_grouped((const UpdateArgs*)b->upd_sweep.tab, b->upd_sweep.offs, b->upd_sweep.n,
                                b->upd_sweep.total, s, ZT_GATE_SWEEP)))
        return rc;
    b->launches++;   // each instance's last CTA takes its stop decision
    return ZT_OK;
}

int enqueue_final(zt_batch* b, cudaStream_t s) {
    int rc;
    if (b->final_mode == ZT_FINAL_FRESH && (rc = enqueue_products(b, s, ZT_GATE_FINAL))) return rc;
    if ((rc = zt_update_grouped((const UpdateArgs*)b->upd_final.tab, b->upd_final.offs, b->upd_final.n,
                                b->upd_final.total, s, ZT_GATE_FINAL)))
        return rc;
    b->launches++;   // each instance's last CTA marks it finalised
    return ZT_OK;
}

int enqueue_read_states(zt_batch* b, cudaStream_t s) {
    state_gather<<<(b->n + 127) / 128, 128, 0, s>>>(b->dstates, b->n, b->gathered);
    int rc = count_launch(b, "state_gather");
    if (rc) return rc;
    ZT_CU(cudaMemcpyAsync(b->hstates, b->gathered, (size_t)b->n * sizeof(zt_dev_state), cudaMemcpyDeviceToHost, s));
    return ZT_OK;
}

int enqueue_first_round(zt_batch* b, double tol, int maxit, int nsweeps, cudaStream_t s) {
    int rc;
    copy_grouped<<<b->copy.total, 256, 0, s>>>((const CopyArgs*)b->copy.tab, b->copy.offs, b->copy.n, tol, maxit);
    if ((rc = count_launch(b, "copy_grouped"))) return rc;
    for (int c = 0; c < nsweeps; ++c)
        if ((rc = enqueue_sweep(b, s))) return rc;
    if ((rc = enqueue_final(b, s))) return rc;
    return enqueue_read_states(b, s);
}

int enqueue_more_round(zt_batch* b, int nsweeps, cudaStream_t s) {
    int rc;
    for (int c = 0; c < nsweeps; ++c)
        if ((rc = enqueue_sweep(b, s))) return rc;
    if ((rc = enqueue_final(b, s))) return rc;
    return enqueue_read_states(b, s);
}

int capture(zt_batch* b, cudaStream_t s, cudaGraphExec_t* out, bool first, double tol, int maxit, int nsweeps) {
    cudaGraph_t g = nullptr;
    ZT_CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const long k0 = b->launches;
    int rc = first ? enqueue_first_round(b, tol, maxit, nsweeps, s) : enqueue_more_round(b, nsweeps, s);
    (first ? b->g_first_k : b->g_more_k) = b->launches - k0;
    b->launches = k0;   // counted when the graph is launched
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return zt_cuda_check(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return zt_cuda_check(e, "cudaGraphInstantiate");
    return ZT_OK;
}

void drop_graphs(zt_batch* b) {
    if (b->g_first) cudaGraphExecDestroy(b->g_first);
    if (b->g_more) cudaGraphExecDestroy(b->g_more);
    b->g_first = b->g_more = nullptr;
    b->g_tol_maxit_set = 0;
}

}  // namespace

extern "C" void zt_batch_destroy(zt_batch* b) {
    if (!b) return;
    // steps end with a host synchronisation; only graph replays on the own
    // stream can still be in flight (no device-wide sync: another thread may
    // be capturing a graph)
    if (b->own) cudaStreamSynchronize(b->own);
    drop_graphs(b);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->own) cudaStreamDestroy(b->own);
    if (b->mstream) {   // every step ended with a host synchronisation: nothing of the batch is in flight
        zt_dfree(b->dbuf, b->mstream);
        zt_dfree(b->dstates, b->mstream);
        zt_dfree(b->gathered, b->mstream);
        cudaStreamDestroy(b->mstream);
    }
    zt_host_states_release(b->hstates, b->n);
    delete b;
}

extern "C" int zt_batch_create(int count, zt_plan* const* plans, double* const* W, const double* h,
                               zt_batch** out) {
    if (!out) return zt_fail(ZT_EINVAL, "zt_batch_create: out is NULL");
    *out = nullptr;
    if (count < 1 || !plans || !W || !h) return zt_fail(ZT_EINVAL, "zt_batch_create: empty batch or NULL array");
    zt_batch* b = new (std::nothrow) zt_batch();
    if (!b) return zt_fail(ZT_ENOMEM, "host allocation failed");
    auto fail = [&](int rc) {
        zt_batch_destroy(b);
        return rc;
    };
    b->n = count;
    {
        cudaError_t e0 = zt_setup_stream(&b->mstream);
        if (e0 != cudaSuccess) return fail(zt_cuda_check(e0, "stream create"));
    }
    int dev = 0;
    cudaGetDevice(&dev);
    b->device = dev;
    for (int i = 0; i < count; ++i) {
        zt_plan* p = plans[i];
        if (!p || !W[i]) return fail(zt_fail(ZT_EINVAL, "zt_batch_create: instance %d has a NULL plan or W", i));
        if (p->N > b->maxN) b->maxN = p->N;
        if (((uintptr_t)W[i]) & 15u) return fail(zt_fail(ZT_EINVAL, "zt_batch_create: W[%d] not 16-byte aligned", i));
        if (!std::isfinite(h[i])) return fail(zt_fail(ZT_EINVAL, "zt_batch_create: h[%d] not finite", i));
        if (p->device != dev) return fail(zt_fail(ZT_EINVAL, "zt_batch_create: plans on different devices"));
        for (int j = 0; j < i; ++j)
            if (plans[j] == p) return fail(zt_fail(ZT_EINVAL, "zt_batch_create: plan %d appears twice", i));
        if (i == 0) b->final_mode = p->tun.final_mode;
        if (p->tun.final_mode != b->final_mode)
            return fail(zt_fail(ZT_EINVAL, "zt_batch_create: instances must share the final mode"));
        // a fixed chunk if any instance asks for one (the smallest), else adaptive
        if (p->tun.sweeps_per_sync > 0 && (b->sweeps_per_sync == 0 || p->tun.sweeps_per_sync < b->sweeps_per_sync))
            b->sweeps_per_sync = p->tun.sweeps_per_sync;
        b->plans.push_back(p);
        b->W.push_back(reinterpret_cast<double2*>(W[i]));
        b->h.push_back(h[i]);
    }
    Builder bl;
    std::vector<CopyArgs> cp;
    std::vector<SolveArgs> sv;
    std::vector<SplitRowsArgs> sP, sW, sA;   // Pt and Wt splits share one table (Pt entries first)
    std::vector<GemmEntry> g1, g2;
    std::vector<Fp64GemmArgs> fa, fb;
    std::vector<UpdateArgs> us, uf;
    std::vector<int> c_cp, c_sv, c_sP, c_g1, c_g2, c_fa, c_fb, c_up;
    int rc;
    for (int i = 0; i < count; ++i) {
        zt_plan* p = plans[i];
        const int N = p->N;
        const long long nn = (long long)N * N;
        cp.push_back({b->W[i], p->Wn, p->Wt, nn, p->state, p->tun.first_iterate == ZT_FIRST_EXTRAPOLATED ? 1 : 0});
        c_cp.push_back((int)((nn + COPY_PER_CTA - 1) / COPY_PER_CTA));
        SolveArgs sa;
        zt_solve_args(p, p->Wt, p->P, &sa);
        sv.push_back(sa);
        c_sv.push_back(zt_solve_ctas(N));
        if (p->precision == ZT_PRECISION_SPLIT) {
            SplitRowsArgs ra;
            if ((rc = zt_split_rows_args(p, p->P, 1, -1, &ra))) return fail(rc);
            sP.push_back(ra);
            if ((rc = zt_split_rows_args(p, p->Wt, 0, 0, &ra))) return fail(rc);
            sW.push_back(ra);
            if ((rc = zt_split_rows_args(p, p->A, 0, 1, &ra))) return fail(rc);
            sA.push_back(ra);
            c_sP.push_back(N);
            GemmEntry e;
            int ctas;
            if ((rc = zt_split_gemm_entry(p, 0, p->A, -1.0, 0, 1, &e, &ctas))) return fail(rc);   // A = Pt Wt
            g1.push_back(e);
            c_g1.push_back(ctas);
            if ((rc = zt_split_gemm_entry(p, 1, p->B, +1.0, 1, 0, &e, &ctas))) return fail(rc);   // B = Pt A^H
            g2.push_back(e);
            c_g2.push_back(ctas);
        } else {
            Fp64GemmArgs f;
            int ctas;
            zt_fp64_gemm_args(p, p->P, p->Wt, p->A, -1.0, 0, &f, &ctas);
            fa.push_back(f);
            c_fa.push_back(ctas);
            zt_fp64_gemm_args(p, p->A, p->P, p->B, -1.0, 1, &f, &ctas);
            fb.push_back(f);
            c_fb.push_back(ctas);
        }
        const double hh = b->h[i];
        UpdateArgs u;
        u.A = p->A;
        u.B = p->B;
        u.h2 = hh / 2.0;
        u.N = N;
        u.st = p->state;
        u.gate = ZT_GATE_NONE;
        u.done = p->upd_done;
        u.nctas = zt_update_ctas(N);
        u.base = p->Wn;   // sweep: Wt <- W_n + h/2 (A - A^H) + h^2/4 B
        u.old = p->Wt;
        u.out = p->Wt;
        u.c2 = hh * hh / 4.0;
        u.partials = p->partials;
        u.final_write = 0;
        us.push_back(u);
        u.base = p->Wt;   // final: W_{n+1} = Wt + h/2 (A - A^H) - h^2/4 B
        u.old = nullptr;
        u.out = b->W[i];
        u.c2 = -hh * hh / 4.0;
        u.partials = nullptr;
        u.final_write = 1;
        uf.push_back(u);
        c_up.push_back(zt_update_ctas(N));
    }
    bl.add(&b->copy, cp, c_cp);
    bl.add(&b->solve, sv, c_sv);
    if (!sP.empty()) {
        std::vector<SplitRowsArgs> sPW(sP);
        sPW.insert(sPW.end(), sW.begin(), sW.end());
        std::vector<int> c_PW(c_sP);
        c_PW.insert(c_PW.end(), c_sP.begin(), c_sP.end());
        bl.add(&b->split_PW, sPW, c_PW);
        bl.add(&b->split_A, sA, c_sP);
        bl.add(&b->gemm1, g1, c_g1);
        bl.add(&b->gemm2, g2, c_g2);
    }
    if (!fa.empty()) {
        bl.add(&b->f64a, fa, c_fa);
        bl.add(&b->f64b, fb, c_fb);
    }
    bl.add(&b->upd_sweep, us, c_up);
    bl.add(&b->upd_final, uf, c_up);
    if ((rc = bl.upload(b))) return fail(rc);
    std::vector<zt_dev_state*> sts(count);
    for (int i = 0; i < count; ++i) sts[i] = plans[i]->state;
    cudaError_t e;
    // a plan whose previous step advanced another W or h has no usable history here
    for (int i = 0; i < count; ++i)
        if (plans[i]->last_W != (const void*)b->W[i] || plans[i]->last_h != b->h[i])
            if ((e = cudaMemsetAsync(&plans[i]->state->hist, 0, sizeof(int), b->mstream)) != cudaSuccess)
                return fail(zt_cuda_check(e, "cudaMemsetAsync(hist)"));
    if ((e = ZT_DMALLOC(b->dstates, count * sizeof(zt_dev_state*), b->mstream)) != cudaSuccess)
        return fail(zt_cuda_check(e, "cudaMallocAsync"));
    if ((e = cudaMemcpyAsync(b->dstates, sts.data(), count * sizeof(zt_dev_state*), cudaMemcpyHostToDevice,
                             b->mstream)) != cudaSuccess)
        return fail(zt_cuda_check(e, "cudaMemcpyAsync"));
    if ((e = ZT_DMALLOC(b->gathered, count * sizeof(zt_dev_state), b->mstream)) != cudaSuccess)
        return fail(zt_cuda_check(e, "cudaMallocAsync"));
    if ((e = cudaStreamSynchronize(b->mstream)) != cudaSuccess) return fail(zt_cuda_check(e, "set-up"));
    b->hstates = zt_host_states_acquire(count);
    if (!b->hstates) return fail(zt_fail(ZT_ENOMEM, "pinned host allocation failed"));
    *out = b;
    return ZT_OK;
}

extern "C" int zt_batch_set_graph(zt_batch* b, int enable) {
    if (!b) return zt_fail(ZT_EINVAL, "batch is NULL");
    if (b->own) ZT_CU(cudaStreamSynchronize(b->own));
    drop_graphs(b);
    b->use_graph = enable ? 1 : 0;
    if (b->use_graph && !b->own) {   // the legacy default stream cannot be captured
        ZT_CU(cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking));
        ZT_CU(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    }
    return ZT_OK;
}

extern "C" long zt_batch_launch_count(const zt_batch* b) { return b ? b->launches : 0; }

static int batch_step_impl(zt_batch* b, double tol, int maxit, zt_step_stats* stats, cudaStream_t s) {
    int rc;
    // sweeps per host check: fixed, or as many as the slowest instance took in the previous step
    const int spc = b->sweeps_per_sync ? b->sweeps_per_sync : (b->last_max > 0 ? b->last_max : 4);
    if (b->use_graph) {   // work goes to the batch's own stream, after what the caller queued on s
        ZT_CU(cudaEventRecord(b->ev_in, s));
        ZT_CU(cudaStreamWaitEvent(b->own, b->ev_in, 0));
        s = b->own;
        if (b->g_tol_maxit_set && (b->g_tol != tol || b->g_maxit != maxit || b->g_stream != s || b->g_spc != spc))
            drop_graphs(b);
        if (!b->g_first) {
            if ((rc = capture(b, s, &b->g_first, true, tol, maxit, spc))) return rc;
            if ((rc = capture(b, s, &b->g_more, false, tol, maxit, spc))) return rc;
            b->g_tol = tol;
            b->g_maxit = maxit;
            b->g_stream = s;
            b->g_spc = spc;
            b->g_tol_maxit_set = 1;
        }
    }
    int enq = 0;
    for (int round = 0;; ++round) {
        const int nsw = (maxit - enq < spc) ? (maxit - enq) : spc;
        if (b->use_graph && nsw == spc) {
            ZT_CU(cudaGraphLaunch(round == 0 ? b->g_first : b->g_more, s));
            b->launches += round == 0 ? b->g_first_k : b->g_more_k;
        } else if (round == 0) {
            if ((rc = enqueue_first_round(b, tol, maxit, nsw, s))) return rc;
        } else {
            if ((rc = enqueue_more_round(b, nsw, s))) return rc;
        }
        enq += nsw;
        ZT_CU(cudaStreamSynchronize(s));
        bool all = true;
        for (int i = 0; i < b->n; ++i) all = all && b->hstates[i].done;
        if (all) break;
        if (enq >= maxit) return zt_fail(ZT_ECUDA, "isomp_step_batched: states not done after maxit sweeps");
    }
    int worst = ZT_OK, most = 0;
    for (int i = 0; i < b->n; ++i) {
        b->plans[i]->last_W = b->W[i];   // the history the next step (batched or not) may use
        b->plans[i]->last_h = b->h[i];
        const zt_dev_state& hs = b->hstates[i];
        if (hs.iters > most && !hs.timeout && !hs.nonfinite) most = hs.iters;
        if (stats) {
            stats[i].iters = hs.iters;
            stats[i].converged = hs.converged;
            stats[i].residual = hs.residual;
        }
        if (hs.timeout) worst = ZT_ETIMEOUT;
        else if (hs.nonfinite && worst != ZT_ETIMEOUT) worst = ZT_ENONFINITE;
        else if (!hs.converged && worst == ZT_OK) worst = ZT_NOT_CONVERGED;
    }
    if (most > 0) b->last_max = most;
    if (worst == ZT_ETIMEOUT) return zt_fail(worst, "isomp_step_batched: a bounded device wait ran out");
    if (worst == ZT_ENONFINITE) return zt_fail(worst, "isomp_step_batched: a residual is not finite");
    if (worst == ZT_NOT_CONVERGED) return zt_fail(worst, "isomp_step_batched: some instances did not converge");
    return ZT_OK;
}

extern "C" int isomp_step_batched(zt_batch* b, double tol, int maxit, zt_step_stats* stats, void* stream) {
    if (!b) return zt_fail(ZT_EINVAL, "batch is NULL");
    if (!(tol >= 0.0)) return zt_fail(ZT_EINVAL, "tol must be >= 0");
    if (maxit < 1 || maxit > 100000) return zt_fail(ZT_EINVAL, "maxit outside [1, 100000]");
    return batch_step_impl(b, tol, maxit, stats, (cudaStream_t)stream);
}

extern "C" int isomp_run_batched(zt_batch* b, long nsteps, double tol, int maxit, zt_run_stats* stats,
                                 void* stream) {
    if (!b) return zt_fail(ZT_EINVAL, "batch is NULL");
    if (nsteps < 0) return zt_fail(ZT_EINVAL, "nsteps < 0");
    std::vector<zt_step_stats> st(b->n);
    zt_run_stats tot{};
    tot.all_converged = 1;
    int worst = ZT_OK;
    for (long k = 0; k < nsteps; ++k) {
        int rc = isomp_step_batched(b, tol, maxit, st.data(), stream);
        if (rc < 0) {
            if (stats) *stats = tot;
            return rc;
        }
        if (rc == ZT_NOT_CONVERGED) worst = rc;
        tot.steps++;
        for (int i = 0; i < b->n; ++i) {
            tot.total_iters += st[i].iters;
            if (st[i].iters > tot.max_iters) tot.max_iters = st[i].iters;
            if (!st[i].converged) tot.all_converged = 0;
            if (st[i].residual > tot.max_residual) tot.max_residual = st[i].residual;
        }
    }
    if (stats) *stats = tot;
    if (worst) return zt_fail(worst, "isomp_run_batched: some instances did not converge");
    return ZT_OK;
}
