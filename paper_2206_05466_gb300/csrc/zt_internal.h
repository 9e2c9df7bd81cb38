// Internal declarations shared by the translation units of libzeitlin.
#pragma once

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
    int    pad0, pad1;
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
    return gate == ZT_GATE_SWEEP ? d != 0 : d == 0;
#else
    (void)st; (void)gate;
    return false;
#endif
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
    double* fac_l = nullptr;   // LDL^T multiplier l_i  (l_0 = 0)
    double* fac_nd = nullptr;  // -1 / d_i              (0 for the dropped m=0 row)
    // Step workspace, complex N x N interleaved.
    double2* Wn = nullptr;
    double2* Wt = nullptr;
    double2* P = nullptr;
    double2* A = nullptr;
    double2* B = nullptr;
    double* partials = nullptr;
    int npartials = 0;
    // segmented stream solve: per-(diagonal, segment) end/start values
    int nseg = 0;
    double2* seg_z = nullptr;
    double* seg_g = nullptr;
    double2* seg_x = nullptr;
    double* seg_h = nullptr;
    double2* sum_x = nullptr;
    double* sum_h = nullptr;
    zt_dev_state* state = nullptr;
    zt_dev_state* h_state = nullptr;   // pinned host mirror
    zt_split_ws* split = nullptr;
    long launches = 0;
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
void zt_solve_destroy(zt_plan* p);
// C = alpha * X conj(Y)^T, FP64 DFMA.  With lower_only, only tiles that
// touch the lower triangle (i >= j) are computed.
int zt_launch_zgemm_fp64(zt_plan* p, const double2* X, const double2* Y, double2* C,
                         double alpha, int lower_only, cudaStream_t s, int gate);
// Split-precision version (tcgen05).  Same contract.
int zt_split_create(zt_plan* p);
void zt_split_destroy(zt_plan* p);
int zt_launch_zgemm_split(zt_plan* p, const double2* X, const double2* Y, double2* C,
                          double alpha, int lower_only, cudaStream_t s, int gate);
// The two halves of the split product: digit splitting of one operand (into
// the X' planes and/or one of two B'^T slots) and the tcgen05 product of the
// X' planes with a B'^T slot.
int zt_split_operand(zt_plan* p, const double2* X, int to_a, int b_slot, cudaStream_t s, int gate);
int zt_split_product(zt_plan* p, int b_slot, double2* C, double alpha, int lower_only, cudaStream_t s, int gate);
