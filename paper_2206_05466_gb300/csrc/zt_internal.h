// Internal declarations shared by the translation units of libzeitlin.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "zeitlin.h"

// Device-resident state of one IsoMP step: the convergence decision of the
// fixed-point iteration lives here so that no host round trip is needed
// between sweeps.
struct zt_dev_state {
    int    done;        // 1 once the sweeps are finished (converged, maxit or non-finite)
    int    iters;       // sweeps completed
    int    converged;   // residual fell below tol
    int    nonfinite;   // residual was NaN/Inf
    int    timeout;     // a bounded device wait ran out (tcgen05 kernels)
    int    maxit;
    int    finalized;   // W_{n+1} has been written (set after the final assembly completed)
    int    hist;        // the plan's W_n buffer holds the previous step's W_n and that step
                        // converged: the next step may start from the extrapolated midpoint
    double residual;    // last Frobenius residual
    double tol;
};

// Gate a kernel on the step state: sweep kernels skip once done, the kernels
// of the final assembly run only once done.
enum zt_gate : int { ZT_GATE_NONE = 0, ZT_GATE_SWEEP = 1, ZT_GATE_FINAL = 2 };

__host__ __device__ inline bool zt_gate_skip(const zt_dev_state* st, int gate) {
#ifdef __CUDA_ARCH__
    if (gate == ZT_GATE_NONE || st == nullptr) return false;
    int d = *(volatile const int*)&st->done;
    if (gate == ZT_GATE_SWEEP) return d != 0;
    return d == 0 || *(volatile const int*)&st->finalized != 0;
#else
    (void)st; (void)gate;
    return false;
#endif
}

// Grouped launches: one grid covers several instances; offs[0..n] are the
// prefix sums of the CTAs each instance needs, and a CTA finds its instance
// by binary search.
__device__ __forceinline__ int zt_group_find(const int* offs, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (offs[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// -x by flipping the sign bit: an integer operation, where a stand-alone FP64
// negation would take an issue slot of the narrow FP64 pipe.
__device__ __forceinline__ double neg(double x) {
    return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}

// First iterate of the fixed point (Eq. 9) from the last two states: the
// midpoint extrapolated along the trajectory, W_n + (W_n - W_{n-1}) / 2, an
// O(h^2) guess of the fixed point where W_n is an O(h) one.  Element-wise and
// odd in (w, wp), so a skew-Hermitian pair gives a skew-Hermitian result.
__device__ __forceinline__ double2 zt_extrapolate(double2 w, double2 wp) {
    return make_double2(fma(0.5, w.x - wp.x, w.x), fma(0.5, w.y - wp.y, w.y));
}

// Packed lower-triangular index of (r, c), c <= r.
__host__ __device__ inline size_t zt_tri(int r, int c) {
    return (size_t)r * (size_t)(r + 1) / 2 + (size_t)c;
}

struct zt_split_ws;   // split-precision workspace (zt_split.cu)

// One timed launch (measurement hook).
struct zt_timer_rec {
    cudaEvent_t a = nullptr, b = nullptr;
    int kind = 0;
    int sweep = -1;       // sweep index inside a step, ZT_SWEEP_FINAL, or -1 outside a step
    double work = 0.0;
    double work_alg = 0.0;
};
constexpr int ZT_SWEEP_FINAL = 1 << 30;

struct zt_plan {
    int N = 0;
    int precision = 0;
    int device = 0;
    zt_tuning tun{};
    // Constant per-diagonal data in packed lower-triangular layout: entry
    // (r, c) belongs to diagonal m = r - c at position i = c.
    double* lap_a = nullptr;   // T_m diagonal a_i
    double* lap_b = nullptr;   // T_m off-diagonal b_i (coupling i, i+1)
    // Step workspace, complex N x N interleaved.
    double2* Wn = nullptr;
    double2* Wt = nullptr;
    double2* P = nullptr;
    double2* A = nullptr;
    double2* B = nullptr;
    double* partials = nullptr;
    double* cas_part = nullptr;   // Casimir partial sums [CTAs + 1][8]
    int npartials = 0;
    // Stream solve by bands of 32 diagonals and segments of 16 rows (zt_solve.cu).
    // Per element, packed lower-triangular row-major (entry (r, c) at zt_tri(r, c)),
    // as pairs so that one 16-byte load brings both numbers a sweep needs:
    double2* fac_lnd = nullptr;   // (-l_i, nd_i): LDL^T multiplier negated (l_0 = 0), nd_i = -1 / d_i
                                  // (0 for the dropped m = 0 row)
    double2* fac_fh = nullptr;    // (F_i, H_i): the segment's responses to its forward and backward inflows
    // Per (segment k, diagonal m), [K][N] (coalesced over m):
    int nseg = 0;              // K = 2 ceil(N / 32) segments of 16 rows
    double2* seg_z = nullptr;  // local forward sweep at the segment's last position
    double2* seg_x = nullptr;  // local backward sweep at the segment's first position
    double* seg_g = nullptr;   // G at the last position (constant)
    double* seg_f = nullptr;   // F at the first position (constant)
    double* seg_h = nullptr;   // H at the first position (constant)
    double2* carry_f = nullptr;   // forward inflow of the segment
    double2* carry_b = nullptr;   // backward inflow of the segment
    double2* sum_x = nullptr;  // [K] m = 0: sum of the local backward sweep over the segment
    double* sum_f = nullptr;   // [K] m = 0: sum of F over the segment (constant)
    double* sum_h = nullptr;   // [K] m = 0: sum of H over the segment (constant)
    double2* sol_mu = nullptr;   // m = 0: mean of the solution before its removal
    zt_dev_state* state = nullptr;
    zt_dev_state* h_state = nullptr;   // pinned host mirror
    unsigned int* upd_done = nullptr;  // finished CTAs of the running update launch
    zt_split_ws* split = nullptr;
    long launches = 0;
    int last_iters = 0;   // sweeps of the previous step (adaptive sweeps_per_sync)
    const void* last_W = nullptr;   // W and h of the plan's previous step (the history of the
    double last_h = 0.0;            // extrapolated first iterate is used only for the same W and h)
    // Device memory of the plan comes from the stream-ordered allocator on a
    // private stream: creating or freeing a plan never synchronises the
    // device (other threads may keep long-running work on it).  Frees are
    // ordered after `last_use`, recorded after every launch sequence.
    cudaStream_t mstream = nullptr;
    cudaEvent_t last_use = nullptr;
    // measurement hook
    int timing = 0;
    unsigned long long* d_units = nullptr;   // MMA units (128 x 256 x 64) issued by split products
    int cur_sweep = -1;
    zt_timer_rec* recs = nullptr;
    int nrecs = 0, caprecs = 0;
    long t_n[ZT_KERNEL_KINDS] = {0, 0, 0, 0};
    double t_ms[ZT_KERNEL_KINDS] = {0, 0, 0, 0};
    double t_work[ZT_KERNEL_KINDS] = {0, 0, 0, 0};
    double t_work_alg[ZT_KERNEL_KINDS] = {0, 0, 0, 0};
};

// Measurement hook: bracket a launch with events when timing is enabled.
int zt_timer_begin(zt_plan* p, int kind, double work, double work_alg, cudaStream_t s);
void zt_timer_end(zt_plan* p, int idx, cudaStream_t s);
// Fold finished records into the totals; iters >= 0 drops sweeps >= iters.
int zt_timer_collect(zt_plan* p, int iters);

// ---- per-instance kernel arguments (one table entry per instance in grouped launches)

struct SolveArgs {     // stream solve (zt_solve.cu)
    const double2* W;
    double2* P;
    const double2* fln;    // packed lower-triangular (-l, nd) pairs (constant)
    const double2* ffh;    // packed lower-triangular (F, H) pairs (constant)
    double2* seg_z;        // [K][N]
    double2* seg_x;        // [K][N]
    const double* seg_g;   // [K][N] (constant)
    const double* seg_f;   // [K][N] (constant)
    const double* seg_h;   // [K][N] (constant)
    double2* cf;           // [K][N] forward inflow (z at the position before the segment)
    double2* cb;           // [K][N] backward inflow (x at the position after the segment)
    double2* sum_x;        // [K] m = 0 only
    const double* sum_f;   // [K] m = 0 only (constant)
    const double* sum_h;   // [K] m = 0 only (constant)
    double2* mu;           // m = 0 only: mean of the solution
    int N, K;
    const zt_dev_state* st;
    int gate;
};

struct SplitRowsArgs { // digit splitting of one operand (zt_split.cu)
    const double2* X;
    int N, s, beta, ldk;
    void* dA;          // __nv_bfloat16 planes [s][Mpad][ldk] or NULL
    int Mpad;
    int* eA;
    void* dB;          // __nv_bfloat16 planes [s][Npad][ldk] or NULL
    int Npad;
    int* eB;
    int* occA;         // [ngA][nkb] or NULL
    int occA_rows, occA_n;
    int* occB;         // [ngB][nkb] or NULL
    int occB_rows, occB_n;
    const zt_dev_state* st;
    int gate;
};

struct SplitArgs {     // tcgen05 split product (zt_split.cu)
    int N, s, beta, ldk, Mpad, Npad, u, exact_groups, ntn, lower_only;
    int s_occA;   // digits X' was split into (the occupancy's reference; s <= s_occA)
    // digit occupancy per (row group, K block): s - (first nonzero digit), 0 = all zero;
    // NULL disables zero-unit skipping
    const int* occA;
    const int* occB;
    unsigned long long* units;   // if not NULL: += MMA units (128 x 256 x 64) issued by each CTA
    int ntng;          // output tiles along the columns of C'
    const int* order;  // launch order of tiles (linear index tig * ntng + tjg)
    int ngroups;       // tiles of the launch
    unsigned long long wait_ns;  // limit of one bounded mbarrier wait
    int stall_loads;   // testing only: > 0 stops the TMA producer after stall_loads - 1 loads
    // The occupancy arrays this product reads are accumulated with atomicMax by the
    // splitter; the launch's last CTA to finish (counted in `done`, nctas CTAs)
    // zeroes them for the next split.  NULL: nothing to clear.
    int* clr_a;
    int clr_a_n;
    int* clr_b;
    int clr_b_n;
    unsigned int* done;
    int nctas;
    unsigned int* tickets;   // persistent form: tile ticket counter, zero at launch
    double alpha;
    const int* eA;
    const int* eB;
    double* C;
    zt_dev_state* st;
    int gate;
};

struct GemmEntry {   // grouped split product: tensor maps live in global memory (aligned like CUtensorMap)
    CUtensorMap tmA;
    CUtensorMap tmB;
    SplitArgs a;
};

struct Fp64GemmArgs {  // FP64 product (zt_fp64.cu)
    const double2* X;
    const double2* Y;
    double2* C;
    double alpha;
    int N, lower_only, gx;   // gx: tiles along columns
    const zt_dev_state* st;
    int gate;
};

struct UpdateArgs {    // fixed-point update / W_{n+1} assembly (zt_plan.cu)
    const double2* base;
    const double2* A;
    const double2* B;
    const double2* old;
    double2* out;
    double h2, c2;
    double* partials;
    int N, final_write;
    zt_dev_state* st;
    int gate;
    // The launch's last CTA to finish (counted in `done`, nctas CTAs) reduces the
    // residual partials and takes the stop decision (sweeps), or marks the state
    // finalised (the W_{n+1} assembly).
    unsigned int* done;
    int nctas;
};

// Plan set-up work goes to a private non-blocking stream of the greatest
// priority, so that it is scheduled ahead of long-running work other threads
// keep on the device.
// Host mirrors of device state records live in a process-wide pinned arena
// (chunks from cudaHostAlloc, kept for the life of the process), so that the
// per-step device-to-host copy of the states is asynchronous.  A copy into
// pageable memory would hold the calling thread inside the driver until its
// stream drained, stalling other threads' driver calls (stream creation,
// allocation) for as long.  Returns nullptr when pinned memory is exhausted.
zt_dev_state* zt_host_states_acquire(int n);
void zt_host_states_release(zt_dev_state* p, int n);

inline cudaError_t zt_setup_stream(cudaStream_t* s) {
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    return cudaStreamCreateWithPriority(s, cudaStreamNonBlocking, greatest);
}

// Kernel attributes (dynamic shared-memory limits) are set once per device
// and process: setting them again while other threads run the kernels is
// unnecessary and can stall.  `bit` names the kernel family.
enum zt_attr_bit : unsigned { ZT_ATTR_SOLVE = 1u, ZT_ATTR_SPLIT = 2u, ZT_ATTR_POOL = 4u };
bool zt_attr_needed(unsigned bit);   // true once per (device, bit); marks it set

// Stream-ordered device allocation on the plan's private stream.
#define ZT_DMALLOC(ptr, bytes, stream) cudaMallocAsync((void**)&(ptr), (bytes), (stream))
inline void zt_dfree(void* ptr, cudaStream_t s) {
    if (ptr) cudaFreeAsync(ptr, s);
}
// Remember the last work enqueued on the plan (frees wait for it).
inline void zt_note_use(zt_plan* p, cudaStream_t s) {
    if (p && p->last_use) cudaEventRecord(p->last_use, s);
}

// ---- error handling ---------------------------------------------------------
int zt_fail(int code, const char* fmt, ...);
int zt_cuda_check(cudaError_t e, const char* what);
#define ZT_CU(call)                                                    \
    do {                                                               \
        cudaError_t _e = (call);                                       \
        if (_e != cudaSuccess) return zt_cuda_check(_e, #call);        \
    } while (0)

// ---- kernels (launchers) ----------------------------------------------------
int zt_launch_laplacian(zt_plan* p, const double2* P, double2* W, cudaStream_t s);
int zt_launch_stream_solve(zt_plan* p, const double2* W, double2* P, cudaStream_t s, int gate);
int zt_solve_create(zt_plan* p);
// Factors (host l and nd, packed lower-triangular) and their segment products
// uploaded to the plan in the solve's layout; waits for its own copies.
int zt_solve_upload_factors(zt_plan* p, const double* host_l, const double* host_nd);
size_t zt_solve_bytes(int N);   // device bytes of the solve workspace
constexpr int ZT_SOLVE_LAUNCHES = 3;
void zt_solve_destroy(zt_plan* p);
// C = alpha * X conj(Y)^T, FP64 DFMA.  With lower_only, only tiles that
// touch the lower triangle (i >= j) are computed.
int zt_launch_zgemm_fp64(zt_plan* p, const double2* X, const double2* Y, double2* C,
                         double alpha, int lower_only, cudaStream_t s, int gate);
// Grouped launches over n instances: tab[i] holds instance i's arguments,
// offs[0..n] (device) the prefix sums of CTAs, `total` = offs[n].
int zt_solve_args(zt_plan* p, const double2* W, double2* P, SolveArgs* out);
int zt_solve_ctas(int N);
int zt_solve_grouped(const SolveArgs* tab, const int* offs, int n, int total, int maxN, cudaStream_t s, int gate);
int zt_split_rows_args(zt_plan* p, const double2* X, int to_a, int b_slot, SplitRowsArgs* out);
int zt_split_rows_grouped(const SplitRowsArgs* tab, const int* offs, int n, int total, cudaStream_t s, int gate);
int zt_split_gemm_entry(zt_plan* p, int b_slot, double2* C, double alpha, int lower_only, int keep_a, GemmEntry* out,
                        int* ctas);
int zt_split_gemm_grouped(const GemmEntry* tab, const int* offs, int n, int total, cudaStream_t s, int gate);
int zt_fp64_gemm_args(zt_plan* p, const double2* X, const double2* Y, double2* C, double alpha, int lower_only,
                      Fp64GemmArgs* out, int* ctas);
int zt_fp64_gemm_grouped(const Fp64GemmArgs* tab, const int* offs, int n, int total, cudaStream_t s, int gate);
int zt_update_ctas(int N);
int zt_update_grouped(const UpdateArgs* tab, const int* offs, int n, int total, cudaStream_t s, int gate);
// Split-precision version (tcgen05).  Same contract.
int zt_split_create(zt_plan* p);
size_t zt_split_bytes(int N, const zt_tuning& t);   // device bytes of the split workspace
void zt_split_destroy(zt_plan* p);
int zt_launch_zgemm_split(zt_plan* p, const double2* X, const double2* Y, double2* C,
                          double alpha, int lower_only, cudaStream_t s, int gate);
// The two halves of the split product: digit splitting of one operand (into
// the X' planes and/or one of two B'^T slots) and the tcgen05 product of the
// X' planes with a B'^T slot.
int zt_split_operand(zt_plan* p, const double2* X, int to_a, int b_slot, cudaStream_t s, int gate);
// Two operands split in one launch: X1 into the X' planes and B'^T slot 1, X2 into slot 0.
int zt_split_operands2(zt_plan* p, const double2* X1, const double2* X2, cudaStream_t s, int gate);
int zt_split_product(zt_plan* p, int b_slot, double2* C, double alpha, int lower_only, int keep_a, cudaStream_t s,
                     int gate);
