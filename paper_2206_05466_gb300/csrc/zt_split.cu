// Split-precision complex product on the 5th-generation tensor cores (tcgen05).
//
// C = alpha * X conj(Y)^T (= alpha' X Y for Y in su(N), Sec. 3.1), emulating
// the FP64 product with BF16 digit slices (an error-free splitting in the
// spirit of Ozaki, Ogita, Oishi & Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59 (2012)):
//
//  1. Real formulation.  With X' the N x 2N real matrix of X's interleaved
//     (re, im) rows, and B'^T the 2N x 2N real matrix whose rows 2j, 2j+1
//     are interleaved(Y[j,:]) and interleaved(i Y[j,:]), the real and
//     imaginary parts of sum_k X[i,k] conj(Y[j,k]) are the dot products of
//     row i of X' with rows 2j and 2j+1 of B'^T, so the interleaved complex
//     result is C' = X' B' (one real product, K' = 2N).
//  2. Splitting.  Each row r of X' (and of B'^T) gets an exponent e_r with
//     max|row| < 2^e_r; every entry becomes the integer
//     round(x 2^(s*beta - 1 - e_r)) written in s balanced base-2^beta digits
//     d_0 .. d_{s-1} (|d| <= 2^(beta-1), exact in BF16).  All integer work.
//  3. Products.  Digit planes are multiplied on tcgen05 (kind::f16, BF16 in,
//     FP32 accumulate in TMEM).  Pairs (p, q) with the same g = p + q share a
//     weight, so they accumulate into one TMEM buffer; pairs with g >= s are
//     dropped (triangular truncation).  The leading `exact_groups` groups are
//     accumulated over K chunks short enough that every FP32 partial sum is an
//     exact integer (< 2^24); the rest run over the whole K.
//  4. Recombination.  Each drained TMEM buffer is converted to int64 and
//     added, shifted by its weight, into an int64 fixed-point accumulator
//     held in the output buffer itself; the last step scales it back to FP64.
//
// Kernel structure (128 x 256 output tiles, 352 threads):
//   warp 0  TMA producer: digit tiles (128 x 64 of X', 256 x 64 of B'^T,
//           128-byte swizzle) into a 4-stage shared-memory ring;
//   warp 1  TMEM allocation and the single MMA-issuing thread;
//   warps 2-9  drain TMEM (double-buffered accumulator) into the int64
//           accumulator, two warps per TMEM lane quadrant (128 columns
//           each); the last drain of a tile adds, scales and stores FP64;
//   warp 10 (persistent form) takes tiles from a ticket counter and fills
//           the tile slots the other roles work through.
// The persistent form keeps one CTA per SM for the whole launch, so one
// tile's last drain overlaps the next tile's MMAs; the one-tile-per-CTA form
// serves grouped launches.  Operand tiles are fetched with plain (unicast)
// TMA loads into each CTA's own shared memory.
// Every mbarrier wait is bounded by a wall-clock limit (a kernel argument);
// on expiry the CTA records a timeout in the step state, stops issuing work,
// waits (bounded) for the copies and MMAs it has already issued, frees its
// TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <algorithm>
#include <vector>

#include "zt_internal.h"

namespace {
constexpr int BM = 128;            // tile rows (X' rows)
constexpr int BN = 256;            // tile cols (B'^T rows = real output columns)
constexpr int BK = 64;             // K per stage: 64 BF16 = 128 bytes per row
constexpr int STAGES = 4;
constexpr int A_TILE = BM * BK * 2;
constexpr int B_TILE = BN * BK * 2;
constexpr int STAGE_BYTES = A_TILE + B_TILE;
constexpr int NDRAIN = 256;        // drain / epilogue threads: 8 warps, two per TMEM lane quadrant
constexpr int NTHREADS = 64 + NDRAIN + 32;   // + producer, MMA and scheduler warps
constexpr int MAX_S = 8;
constexpr int NBUF = 2;            // TMEM accumulator buffers per CTA (drain of one overlaps MMAs into the other)
constexpr int CTAS_PER_SM = 1;     // resident CTAs per SM the launch bounds ask for
constexpr uint32_t TMEM_COLS = NBUF * BN;   // 128 x 256 FP32 accumulators
constexpr int MAX_KB = 512;        // K blocks of 64 for N <= 16384
constexpr int EXP_NAN = 0x7fff;    // row exponent marking a non-finite entry
constexpr unsigned long long SETTLE_NS = 2000000000ull;   // teardown waits for issued work: 2 s

// instruction descriptor, kind::f16: D F32, A/B BF16, K-major, M=128, N=256
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                           ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}  // namespace

struct zt_split_ws {
    int s = 7, beta = 7, exact_groups = 4;
    int s2 = 7, u2 = 0;                           // digits of B'^T slot 1 and of the products that
                                                  // read it; accumulator shift for s2 digits
    unsigned long long wait_ns = 2000000000ull;   // limit of one mbarrier wait
    int stall_loads = 0;                          // testing only (zt_tuning.debug_stall_loads)
    int ldk = 0, Mpad = 0, Npad = 0, u = 0;
    __nv_bfloat16* dA = nullptr;   // [s][Mpad][ldk]
    __nv_bfloat16* dB[2] = {nullptr, nullptr};   // two B'^T slots, each [s][Npad][ldk]
    int* eA = nullptr;                           // [Mpad]
    int* eB[2] = {nullptr, nullptr};             // [Npad]
    int nkb = 0, ngA = 0, ngB = 0;               // K blocks; row groups of X'; column groups of B'^T
    int* order_full = nullptr;                   // tile-group launch orders (device), near-diagonal first
    int* order_lower = nullptr;
    int n_full = 0, n_lower = 0;
    int skip_zero = 1;                           // skip digit-pair units whose tiles are all zero
    int persistent = 1;                          // persistent product kernel
    int persistent2 = 1;                         // ... for the products with slot 1 (the second product)
    int nsm = 0;                                 // SMs of the device
    unsigned int* tickets = nullptr;             // tile ticket counter of the persistent kernel,
                                                 // then the count of finished CTAs (occupancy clear)
    int* occA = nullptr;                         // [ngA][nkb]
    int* occB[2] = {nullptr, nullptr};           // [ngB][nkb]
    CUtensorMap tmA, tmB[2];
};


// ---------------------------------------------------------------------------
// device helpers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity: false once another role
// has aborted the CTA or after limit_ns of wall-clock time (which aborts it).
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > limit_ns) {
            *abort_flag = 1;
            return false;
        }
    }
}
// Teardown wait for work this CTA has already issued (copies, MMAs): it
// completes on its own, so the wait ignores the abort flag; bounded all the same.
__device__ bool mbar_settle(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (gtimer() - t0 > SETTLE_NS) return false;
    }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand tile with 128-byte swizzle: rows of 128 B, 8-row atoms of 1 KiB.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused for SW128 K-major)
    d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: 8-row atom
    d |= (uint64_t)1 << 46;                      // descriptor version (sm_100 family)
    d |= (uint64_t)2 << 61;                      // SWIZZLE_128B
    return d;
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// Asynchronous bulk reduce-add of `bytes` (a multiple of 16) of int64 from
// shared to global memory; the L2 performs the additions.
__device__ __forceinline__ void bulk_reduce_add_s64(long long* gdst, uint32_t ssrc, int bytes) {
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u64 [%0], [%1], %2;" ::"l"(gdst), "r"(ssrc),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}


// ---------------------------------------------------------------------------
// Splitting: one CTA per row of X (complex, N entries).  Writes X' digits
// (mode A) and/or the two B'^T rows 2j, 2j+1 built from row j (mode B).
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long to_fixed(double x, int e, int sb) {
    const long long bits = __double_as_longlong(x);
    const int ef = (int)((bits >> 52) & 0x7FF);
    long long mant = bits & 0xFFFFFFFFFFFFFLL;
    int ex;
    if (ef == 0) {
        ex = -1074;
    } else {
        mant |= (1LL << 52);
        ex = ef - 1075;
    }
    const int sh = ex + sb - 1 - e;   // <= sb - 54 for |x| < 2^e
    long long v;
    if (sh >= 0)
        v = mant << sh;
    else if (sh < -62)
        v = 0;
    else
        v = (mant + (1LL << (-sh - 1))) >> (-sh);
    return bits < 0 ? -v : v;
}

__device__ __noinline__ double fixed_to_double_slow(long long v, int E) { return ldexp((double)v, E); }

// v * 2^E rounded to the nearest double (ties to even) with integer operations
// only (the FP64 pipe is narrow); the same value as (double)v * 2^E.  Results
// outside the normal range take the FP64 route.
__device__ __forceinline__ double fixed_to_double(long long v, int E) {
    if (v == 0) return 0.0;
    const unsigned long long sign = (unsigned long long)v & 0x8000000000000000ull;
    const unsigned long long u = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int nb = 64 - __clzll((long long)u);   // significant bits
    int ex = E + nb - 1;                           // unbiased exponent of the result
    unsigned long long m;
    if (nb <= 53) {
        m = u << (53 - nb);
    } else {
        const int r = nb - 53;
        m = u >> r;
        const unsigned long long rem = u & ((1ull << r) - 1), half = 1ull << (r - 1);
        if (rem > half || (rem == half && (m & 1ull))) {
            ++m;
            if (m == (1ull << 53)) {
                m >>= 1;
                ++ex;
            }
        }
    }
    if (ex < -1022 || ex > 1023) return fixed_to_double_slow(v, E);
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)(ex + 1023) << 52) | (m & ((1ull << 52) - 1))));
}

__device__ __forceinline__ void split_rows_body(const SplitRowsArgs& ra, int j) {
    if (zt_gate_skip(ra.st, ra.gate)) return;
    const double2* __restrict__ X = ra.X;
    const int N = ra.N, s = ra.s, beta = ra.beta, ldk = ra.ldk, Mpad = ra.Mpad, Npad = ra.Npad;
    __nv_bfloat16* __restrict__ dA = static_cast<__nv_bfloat16*>(ra.dA);
    __nv_bfloat16* __restrict__ dB = static_cast<__nv_bfloat16*>(ra.dB);
    int* __restrict__ eA = ra.eA;
    int* __restrict__ eB = ra.eB;
    int* __restrict__ occA = ra.occA;
    int* __restrict__ occB = ra.occB;
    const int occA_rows = ra.occA_rows, occB_rows = ra.occB_rows;
    const double2* row = X + (size_t)j * N;
    __shared__ int smax[256];
    int mx = 0;
    for (int k = threadIdx.x; k < N; k += 256) {
        const double2 v = row[k];
        const int e1 = (int)((__double_as_longlong(v.x) >> 52) & 0x7FF);
        const int e2 = (int)((__double_as_longlong(v.y) >> 52) & 0x7FF);
        mx = max(mx, max(e1, e2));
    }
    smax[threadIdx.x] = mx;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) smax[threadIdx.x] = max(smax[threadIdx.x], smax[threadIdx.x + w]);
        __syncthreads();
    }
    mx = smax[0];
    const bool bad = (mx == 0x7FF);
    const int e = max(mx, 1) - 1022;   // max |entry| < 2^e
    const int sb = s * beta;
    const long long R = 1LL << beta, H = R >> 1;
    const size_t planeA = (size_t)Mpad * ldk, planeB = (size_t)Npad * ldk;
    // each thread: 4 consecutive complex entries -> one 16-byte store per plane and row;
    // 8 consecutive threads cover one K block of 64 reals (occupancy reduced by shuffles)
    const int nkb = ldk / 64;
    const int iters = (ldk / 8 + 255) / 256;
    for (int it = 0; it < iters; ++it) {
        const int kq = threadIdx.x + 256 * it;
        const bool live = kq < ldk / 8;
        int fz = s;   // first nonzero digit of this thread's entries (s: none)
        // The fixed-point value v (up to 62 bits) in two 32-bit halves: lo = v mod
        // 2^(kl beta) and hi = v >> (kl beta).  The balanced chain below takes the low
        // kl digits from lo; what is left of lo then is the carry, 0 or 1, into hi,
        // and (hi R^kl + lo + H) >> beta = hi R^(kl-1) + ((lo + H) >> beta), so the
        // digits are those of the chain on v itself, with 32-bit integer operations.
        // (Both halves keep a bit of headroom: kl beta <= 30 and (s - kl) beta <= 30; wider
        // splits, beyond the tuned ones, run the chain on the 64-bit value.)
        const int kl = min(30 / beta, s - 1);
        const bool halves = (s - kl) * beta <= 30;
        long long vr[4], vi[4];
        int lr[4], li[4], hr[4], hi[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = 4 * kq + u;
            vr[u] = vi[u] = 0;
            if (live && k < N && !bad) {
                const double2 v = row[k];
                vr[u] = to_fixed(v.x, e, sb);
                vi[u] = to_fixed(v.y, e, sb);
            }
            const long long m = (1LL << (kl * beta)) - 1;
            lr[u] = (int)(vr[u] & m);
            li[u] = (int)(vi[u] & m);
            hr[u] = (int)(vr[u] >> (kl * beta));
            hi[u] = (int)(vi[u] >> (kl * beta));
        }
        const int Hh = (int)H, Rm = (int)(R - 1);
        // digit p of the four entries from the halves x (lo or hi), stored to the planes
        auto emit = [&](int p, auto* xr, auto* xi) {   // int (a half) or long long (the value)
            __align__(16) __nv_bfloat162 wa[4], wb1[4];
            bool nz = false;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                // balanced digit d = ((v + H) mod R) - H, and (v - d) / R = (v + H) >> beta;
                // digits fit 32 bits, so the conversions stay off the FP64 pipe
                int dr, di;
                if (p > 0) {
                    const auto tr = xr[u] + Hh, ti = xi[u] + Hh;
                    dr = ((int)tr & Rm) - Hh;
                    di = ((int)ti & Rm) - Hh;
                    xr[u] = tr >> beta;
                    xi[u] = ti >> beta;
                } else {
                    dr = (int)xr[u];
                    di = (int)xi[u];
                }
                nz |= (dr | di) != 0;
                const float fr = (float)dr, fi = (float)di;
                // X' row and B'^T row 2j: interleaved(y); B'^T row 2j+1: interleaved(i y) = (-im, re)
                wa[u] = __floats2bfloat162_rn(fr, fi);
                wb1[u] = __floats2bfloat162_rn(-fi, fr);
            }
            if (nz) fz = p;
            if (!live) return;
            const size_t col = (size_t)8 * kq;
            if (dA) *reinterpret_cast<uint4*>(dA + p * planeA + (size_t)j * ldk + col) = *reinterpret_cast<uint4*>(wa);
            if (dB) {
                *reinterpret_cast<uint4*>(dB + p * planeB + (size_t)(2 * j) * ldk + col) = *reinterpret_cast<uint4*>(wa);
                *reinterpret_cast<uint4*>(dB + p * planeB + (size_t)(2 * j + 1) * ldk + col) =
                    *reinterpret_cast<uint4*>(wb1);
            }
        };
        if (halves) {
            for (int p = s - 1; p >= s - kl; --p) emit(p, lr, li);   // the low kl digits from lo
#pragma unroll
            for (int u = 0; u < 4; ++u) {   // lo's carry into hi
                hr[u] += lr[u];
                hi[u] += li[u];
            }
            for (int p = s - kl - 1; p >= 0; --p) emit(p, hr, hi);
        } else {
            for (int p = s - 1; p >= 0; --p) emit(p, vr, vi);
        }
        int occ = s - fz;   // 0: all digits zero, s: leading digit present
        occ = max(occ, __shfl_xor_sync(0xffffffffu, occ, 1));
        occ = max(occ, __shfl_xor_sync(0xffffffffu, occ, 2));
        occ = max(occ, __shfl_xor_sync(0xffffffffu, occ, 4));
        if (live && (kq & 7) == 0) {
            const int kb = kq >> 3;
            if (occA) atomicMax(&occA[(size_t)(j / occA_rows) * nkb + kb], occ);
            if (occB) atomicMax(&occB[(size_t)(j / occB_rows) * nkb + kb], occ);
        }
    }
    if (threadIdx.x == 0) {
        const int ee = bad ? EXP_NAN : e;
        if (eA) eA[j] = ee;
        if (eB) {
            eB[2 * j] = ee;
            eB[2 * j + 1] = ee;
        }
    }
}

__global__ void __launch_bounds__(256) split_rows_kernel(const SplitRowsArgs a) { split_rows_body(a, blockIdx.x); }

// Grouped: one CTA per row of every instance.
__global__ void __launch_bounds__(256) split_rows_grouped(const SplitRowsArgs* tab, const int* offs, int n, int gate) {
    const int inst = zt_group_find(offs, n, blockIdx.x);
    SplitRowsArgs a = tab[inst];
    a.gate = gate;
    split_rows_body(a, blockIdx.x - offs[inst]);
}

// Accumulation segments are counted in issued MMA units (one digit pair on
// one K block of 64): a leading (exact) group may sum at most
// 2^(26 - 2 beta) / 64 units in FP32 before it must be drained, so that every
// partial sum stays an exact integer; later groups run to the end.  Units
// skipped because they are all zero do not count, so sparse tiles drain
// rarely.
__device__ __forceinline__ int seg_units(int g, int beta, int exact_groups) {
    if (g >= exact_groups) return 0x7fffffff;
    const int lim = (1 << (26 - 2 * beta)) / BK;
    return lim < 1 ? 1 : lim;
}
// ---------------------------------------------------------------------------
// The tcgen05 product kernel.
// ---------------------------------------------------------------------------
// Per-tile data shared by the roles: tile-group coordinates, digit occupancy of
// the group's rows of X' (fa) and B'^T (fb) per K block, active units per digit
// group and the number of accumulation segments of the tile.
struct TileSlot {
    int valid;   // 0: no further tile (persistent kernel)
    int tig, tjg;
    int total;
    int gunits[MAX_S];
    uint8_t fa[MAX_KB];   // the unit (p, q, kb) is all zero unless p >= fa[kb] and q >= fb[kb]
    uint8_t fb[MAX_KB];
    // bit kb of amask[g] is set when K block kb has a unit in digit group g
    // (fa[kb] + fb[kb] <= g), so the producer visits only those blocks
    uint32_t amask[MAX_S][MAX_KB / 32];
};
constexpr int TSLOTS = 2;   // tile slots of the persistent kernel (one being worked, one being filled)
// Drain staging: per drain thread one 64-byte slot (8 int64) for the bulk
// reduce-adds of intermediate segments (a 16-column chunk goes out in two
// halves); an 80-byte stride keeps the 16-byte shared stores of a quarter-warp
// on distinct banks.  Small, so that the operand ring has four stages.
constexpr int STG_STRIDE = 80;
constexpr size_t SMEM_BYTES = 1024 /*align slack*/ + (size_t)STAGES * STAGE_BYTES + 256 /*barriers*/ +
                              TSLOTS * sizeof(TileSlot) + (size_t)NDRAIN * STG_STRIDE;

struct SmemMap {
    uint8_t* sA;
    uint8_t* sB;
    uint64_t* full;     // [STAGES] operand stage loaded
    uint64_t* empty;    // [STAGES] operand stage consumed
    uint64_t* accf;     // [NBUF] accumulator segment complete
    uint64_t* acce;     // [NBUF] accumulator buffer drained
    uint64_t* tfull;    // [TSLOTS] tile slot filled
    uint64_t* tempty;   // [TSLOTS] tile slot released
    uint64_t* drain;    // all MMAs retired
    uint32_t* tmem_slot;
    volatile int* abort_flag;
    TileSlot* slots;
    uint8_t* stg;       // [NDRAIN][STG_STRIDE] drain staging
};

__device__ __forceinline__ SmemMap smem_map() {
    extern __shared__ uint8_t smem_raw[];
    SmemMap m;
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    m.sA = base;
    m.sB = base + STAGES * A_TILE;
    m.full = reinterpret_cast<uint64_t*>(m.sB + STAGES * B_TILE);
    m.empty = m.full + STAGES;
    m.accf = m.empty + STAGES;
    m.acce = m.accf + NBUF;
    m.tfull = m.acce + NBUF;
    m.tempty = m.tfull + TSLOTS;
    m.drain = m.tempty + TSLOTS;
    m.tmem_slot = reinterpret_cast<uint32_t*>(m.drain + 1);
    m.abort_flag = reinterpret_cast<volatile int*>(m.tmem_slot + 1);
    m.slots = reinterpret_cast<TileSlot*>(reinterpret_cast<uint8_t*>(m.full) + 256);
    m.stg = reinterpret_cast<uint8_t*>(m.slots + TSLOTS);
    return m;
}

// Tile of a linear launch index; false when it has no element in the
// requested (lower) triangle.
__device__ __forceinline__ bool tile_group(const SplitArgs& a, int grp, int& tig, int& tjg) {
    if (a.order) {   // explicit order (only tiles that have work are listed)
        const int gl = a.order[grp];
        tig = gl / a.ntng;
        tjg = gl % a.ntng;
        return true;
    }
    tig = grp / a.ntng;
    tjg = grp % a.ntng;
    // a 128 x 256 tile of C' covers complex columns [128 tjg, 128 tjg + 128)
    return !(a.lower_only && tjg * (BN / 2) >= (tig + 1) * BM);
}

// One warp fills a tile slot: occupancy, active units per group, segments.
__device__ __forceinline__ void fill_slot_warp(const SplitArgs& a, TileSlot& ts, int tig, int tjg, int nkb, int lane) {
    int u[MAX_S];
#pragma unroll
    for (int g = 0; g < MAX_S; ++g) u[g] = 0;
    for (int kb0 = 0; kb0 < nkb; kb0 += 32) {   // nkb is a multiple of 32 or below it: whole warp iterates
        const int kb = kb0 + lane;
        int c = 2 * MAX_S;   // no unit
        if (kb < nkb) {
            const int fa = a.occA ? a.s_occA - a.occA[(size_t)tig * nkb + kb] : 0;   // may exceed a.s
            const int fb = a.occB ? a.s - a.occB[(size_t)tjg * nkb + kb] : 0;
            ts.fa[kb] = (uint8_t)fa;
            ts.fb[kb] = (uint8_t)fb;
            c = fa + fb;
        }
#pragma unroll
        for (int g = 0; g < MAX_S; ++g) {
            u[g] += max(0, g - c + 1);
            const uint32_t bits = __ballot_sync(0xffffffffu, c <= g);
            if (lane == 0) ts.amask[g][kb0 >> 5] = bits;
        }
    }
    int total = 0;
#pragma unroll
    for (int g = 0; g < MAX_S; ++g) {
        int v = u[g];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (g < a.s) {
            if (lane == 0) ts.gunits[g] = v;
            total += v == 0 ? 0 : (v - 1) / seg_units(g, a.beta, a.exact_groups) + 1;
        }
    }
    if (lane == 0) {
        ts.tig = tig;
        ts.tjg = tjg;
        ts.total = total;
        ts.valid = 1;
    }
    __threadfence_block();
    __syncwarp();
}

// The two last digit groups (s-2, s-1) are accumulated in one K sweep, into the
// two TMEM buffers, when both are inexact (one segment each over the whole K)
// and the tile has units in both: the units of group s-1 at a K block are the
// stages (A_{fa+j}, B_{s-1-fa-j}), j = 0 .. n-1, and the unit j-1 of group s-2,
// (A_{fa+j-1}, B_{s-1-fa-j}), takes the A tile of stage j-1 and the B tile of
// stage j, so group s-2 needs no operand loads of its own.  Each accumulator
// still receives its units in the same order (K blocks ascending, p ascending):
// the result is bitwise the same as sweeping the groups one after the other.
// The two accumulators are then drained together, summed in registers: one
// drain pass for both groups, and no trip through the int64 accumulator in
// global memory when they are the tile's only groups.
__device__ __forceinline__ bool dual_tile(const SplitArgs& a, const TileSlot& ts) {
    return a.s >= 3 && a.exact_groups <= a.s - 2 && ts.gunits[a.s - 2] > 0;
}

// ---- TMA producer (one thread): digit tiles of every active unit of the tile ----
// nload counts the loads issued over the launch (for the teardown).  Returns
// false when the CTA aborted or the testing stall stopped the producer.
__device__ __forceinline__ bool produce_tile(const SplitArgs& a, const TileSlot& ts, const SmemMap& m,
                                             const CUtensorMap* tmA_p, const CUtensorMap* tmB_p, int i0, int c0,
                                             int nkb, int& stage, uint32_t& ph, long long& nload) {
    const int nw = (nkb + 31) >> 5;
    const bool dual = dual_tile(a, ts);
    for (int g = 0; g < a.s; ++g) {
        if (dual && g == a.s - 2) continue;   // its operands come with group s-1's stages
        for (int wi = 0; wi < nw; ++wi)
            for (uint32_t bits = ts.amask[g][wi]; bits; bits &= bits - 1) {
              const int kb = (wi << 5) + __ffs(bits) - 1;
              const int p1 = g - ts.fb[kb];
              for (int p = ts.fa[kb]; p <= p1; ++p) {
                // testing only: stop issuing so that the consumers' bounded waits run out
                if (a.stall_loads > 0 && nload >= a.stall_loads - 1) return false;
                if (!mbar_wait(&m.empty[stage], ph ^ 1, m.abort_flag, a.wait_ns)) return false;
                mbar_expect_tx(&m.full[stage], STAGE_BYTES);
                tma_load_2d(m.sA + stage * A_TILE, tmA_p, &m.full[stage], kb * BK, p * a.Mpad + i0);
                tma_load_2d(m.sB + stage * B_TILE, tmB_p, &m.full[stage], kb * BK, (g - p) * a.Npad + c0);
                ++nload;
                if (++stage == STAGES) {
                    stage = 0;
                    ph ^= 1;
                }
              }
            }
    }
    return true;
}

// Before the CTA leaves: the last STAGES loads issued may still be landing
// (after an abort nobody consumed them).  Load j went to stage j % STAGES as
// phase j / STAGES; earlier loads have completed, because the load j + STAGES
// into the same stage was issued only after the MMA consumed load j.
__device__ __forceinline__ void producer_settle(const SmemMap& m, long long nload) {
    for (long long j = nload > STAGES ? nload - STAGES : 0; j < nload; ++j)
        mbar_settle(&m.full[j % STAGES], (uint32_t)((j / STAGES) & 1));
}

// ---- MMA issuer (one thread): one accumulation segment per exactness budget ----
// stage/ph/seg continue from tile to tile; seg numbers the accumulator buffers.
__device__ __forceinline__ bool mma_tile(const SplitArgs& a, const TileSlot& ts, const SmemMap& m, uint32_t tmem,
                                         int nkb, int& stage, uint32_t& ph, int& seg, unsigned long long& issued) {
    // The units of a digit group arrive in the producer's order; the MMA thread
    // needs only how many there are (the stage ring says where each one is).
    const bool dual = dual_tile(a, ts);
    for (int g = 0; g < a.s; ++g) {
        if (dual && g == a.s - 2) break;   // the last two groups together, below
        const int ulim = seg_units(g, a.beta, a.exact_groups);
        const int nunits = ts.gunits[g];
        int cnt = 0, b = 0;
        bool open = false;
        uint32_t d = 0;
        {
            for (int un = 0; un < nunits; ++un) {
                if (!open) {   // next accumulation segment: wait for its TMEM buffer to be drained
                    b = seg % NBUF;
                    const int use = seg / NBUF;
                    ++seg;
                    if (!mbar_wait(&m.acce[b], (use & 1) ^ 1, m.abort_flag, a.wait_ns)) return false;
                    tc_fence_after();
                    d = tmem + (uint32_t)(b * BN);
                    open = true;
                    cnt = 0;
                }
                if (!mbar_wait(&m.full[stage], ph, m.abort_flag, a.wait_ns)) return false;
                tc_fence_after();
                const uint64_t ad = sw128_desc(smem_u32(m.sA + stage * A_TILE));
                const uint64_t bd = sw128_desc(smem_u32(m.sB + stage * B_TILE));
#pragma unroll
                for (int k = 0; k < BK / 16; ++k)
                    umma_bf16(d, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), (cnt == 0 && k == 0) ? 0u : 1u);
                ++cnt;
                ++issued;
                umma_commit(&m.empty[stage]);
                if (++stage == STAGES) {
                    stage = 0;
                    ph ^= 1;
                }
                if (cnt == ulim) {   // exactness budget of this segment used up
                    umma_commit(&m.accf[b]);
                    open = false;
                }
            }
        }
        if (open) umma_commit(&m.accf[b]);
    }
    if (!dual) return true;
    // groups s-2 (buffer b0) and s-1 (buffer b1) in one sweep over the K blocks of group s-1
    const int b0 = seg % NBUF, use0 = seg / NBUF;
    ++seg;
    if (!mbar_wait(&m.acce[b0], (use0 & 1) ^ 1, m.abort_flag, a.wait_ns)) return false;
    const int b1 = seg % NBUF, use1 = seg / NBUF;
    ++seg;
    if (!mbar_wait(&m.acce[b1], (use1 & 1) ^ 1, m.abort_flag, a.wait_ns)) return false;
    tc_fence_after();
    const uint32_t d0 = tmem + (uint32_t)(b0 * BN), d1 = tmem + (uint32_t)(b1 * BN);
    bool fresh0 = true, fresh1 = true;
    const int nw = (nkb + 31) >> 5, gl = a.s - 1;
    for (int wi = 0; wi < nw; ++wi)
        for (uint32_t bits = ts.amask[gl][wi]; bits; bits &= bits - 1) {
            const int kb = (wi << 5) + __ffs(bits) - 1;
            const int n = gl - ts.fa[kb] - ts.fb[kb] + 1;   // units of group s-1 here (>= 1)
            int pstage = 0;
            uint64_t pad = 0;
            for (int j = 0; j < n; ++j) {
                if (!mbar_wait(&m.full[stage], ph, m.abort_flag, a.wait_ns)) return false;
                tc_fence_after();
                const uint64_t ad = sw128_desc(smem_u32(m.sA + stage * A_TILE));
                const uint64_t bd = sw128_desc(smem_u32(m.sB + stage * B_TILE));
#pragma unroll
                for (int k = 0; k < BK / 16; ++k)
                    umma_bf16(d1, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), (fresh1 && k == 0) ? 0u : 1u);
                fresh1 = false;
                ++issued;
                if (j > 0) {   // group s-2: the previous stage's A with this stage's B
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k)
                        umma_bf16(d0, pad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), (fresh0 && k == 0) ? 0u : 1u);
                    fresh0 = false;
                    ++issued;
                    umma_commit(&m.empty[pstage]);   // the previous stage has no further use
                }
                pstage = stage;
                pad = ad;
                if (++stage == STAGES) {
                    stage = 0;
                    ph ^= 1;
                }
            }
            umma_commit(&m.empty[pstage]);   // the K block's last stage
        }
    umma_commit(&m.accf[b0]);
    umma_commit(&m.accf[b1]);
    return true;
}

// After the MMA thread's last issue (or an abort): every MMA it issued retires
// before TMEM is released or the CTA leaves.
__device__ __forceinline__ void mma_settle(const SmemMap& m, const SplitArgs& a, unsigned long long issued) {
    if (a.units) atomicAdd(a.units, issued);
    umma_commit(m.drain);
    if (!mbar_settle(m.drain, 0)) *m.abort_flag = 1;
}

// ---- drain / epilogue (the 8 drain warps): every segment of the tile into the
// int64 accumulator held in C; the tile's last segment adds, scales and stores
// FP64 in place.  seg continues from tile to tile.
__device__ __forceinline__ bool drain_tile(const SplitArgs& a, const TileSlot& ts, const SmemMap& m, uint32_t tmem,
                                           int i0, int c0, int warp, int lane, int& seg) {
    const int wq = warp & 3;                 // TMEM lane quadrant this warp may access
    const int half = (warp - 2) >> 2;        // column half of the tile this warp drains
    const int gi = i0 + wq * 32 + lane;
    const bool row_ok = gi < a.N;
    const int ncols = 2 * a.N;
    const uint32_t lane_base = (uint32_t)(wq * 32) << 16;
    long long* Crow = reinterpret_cast<long long*>(a.C) + (size_t)gi * ncols;
    const int total = ts.total;
    // FP32 segment sums are integers below 2^31 unless K' and the digits are large
    const bool fits32 = (double)a.s * (double)ncols * (double)(1LL << (2 * a.beta - 2)) < 2147483647.0;
    const bool v32 = (a.N & 1) == 0 && ((uintptr_t)a.C & 31) == 0;   // rows start on 32-byte boundaries
    const int ea = row_ok ? a.eA[gi] : 0;
    const int eoff = -(a.s + 1) * a.beta + 2 + a.u;
    // alpha = +-2^k (the usual +-1) folds into the exponent and the sign
    const long long abits = __double_as_longlong(a.alpha);
    const int aef = (int)((abits >> 52) & 0x7FF);
    const bool apow2 = (abits & 0xFFFFFFFFFFFFFLL) == 0 && aef != 0 && aef != 0x7FF;
    const int aexp = apow2 ? aef - 1023 : 0;
    const unsigned long long asign = apow2 ? ((unsigned long long)abits & 0x8000000000000000ull) : 0ull;
    // staging slot of this thread for the bulk reduce-adds of intermediate segments
    uint8_t* stg = m.stg + (size_t)(threadIdx.x - 64) * STG_STRIDE;
    int nstg = 0;   // bulk operations issued by this thread in this tile
    int tseg = 0;   // segments of this tile drained so far
    const bool dual = dual_tile(a, ts);
    const int tot = dual ? total - 1 : total;   // the last two groups drain as one segment
    for (int g = 0; g < a.s; ++g) {
        const bool pair = dual && g == a.s - 2;   // groups s-2 and s-1, buffers b and b2
        const int ulim = seg_units(g, a.beta, a.exact_groups);
        const int units = ts.gunits[g];
        const int nsegs = pair ? 1 : (units == 0 ? 0 : (units - 1) / ulim + 1);
        const int sh = (a.s - 1 - g) * a.beta - a.u;
        const int sh2 = -a.u;   // weight of group s-1
        for (int q = 0; q < nsegs; ++q) {
            const int b = seg % NBUF, use = seg / NBUF;
            ++seg;
            if (!mbar_wait(&m.accf[b], use & 1, m.abort_flag, a.wait_ns)) {
                if (nstg) bulk_wait_all();
                return false;
            }
            int b2 = 0;
            if (pair) {
                b2 = seg % NBUF;
                const int use2 = seg / NBUF;
                ++seg;
                if (!mbar_wait(&m.accf[b2], use2 & 1, m.abort_flag, a.wait_ns)) {
                    if (nstg) bulk_wait_all();
                    return false;
                }
            }
            tc_fence_after();
            const bool first = tseg == 0, last = tseg == tot - 1;
            ++tseg;
            if (last && nstg) {   // every reduce-add of this tile has landed and is visible
                bulk_wait_all();
                fence_proxy_async_global();
            }
#pragma unroll 1
            for (int ch = 0; ch < BN / 32; ++ch) {   // 16 columns at a time
                const int col0 = half * (BN / 2) + ch * 16;
                uint32_t r[16], r2[16];
                tmem_ld16(tmem + lane_base + (uint32_t)(b * BN + col0), r);
                if (pair) tmem_ld16(tmem + lane_base + (uint32_t)(b2 * BN + col0), r2);
                const int cb = c0 + col0;
                if (!row_ok || cb >= ncols) continue;
                const int lim = min(16, ncols - cb);   // even; a multiple of 4 when v32
                long long v[16];
                // separate loops: a select between the two conversions would run the
                // 64-bit one (FP64 pipe) for every value
                if (fits32) {
#pragma unroll
                    for (int t = 0; t < 16; ++t) v[t] = (long long)__float2int_rn(__uint_as_float(r[t]));
                } else {
#pragma unroll
                    for (int t = 0; t < 16; ++t) v[t] = __float2ll_rn(__uint_as_float(r[t]));
                }
                if (sh >= 0) {
#pragma unroll
                    for (int t = 0; t < 16; ++t) v[t] <<= sh;
                } else {
#pragma unroll
                    for (int t = 0; t < 16; ++t) v[t] = (v[t] + (1LL << (-sh - 1))) >> (-sh);
                }
                if (pair) {   // group s-1 from the second buffer, at its own weight
                    long long v2[16];
                    if (fits32) {
#pragma unroll
                        for (int t = 0; t < 16; ++t) v2[t] = (long long)__float2int_rn(__uint_as_float(r2[t]));
                    } else {
#pragma unroll
                        for (int t = 0; t < 16; ++t) v2[t] = __float2ll_rn(__uint_as_float(r2[t]));
                    }
                    if (sh2 >= 0) {
#pragma unroll
                        for (int t = 0; t < 16; ++t) v[t] += v2[t] << sh2;
                    } else {
#pragma unroll
                        for (int t = 0; t < 16; ++t) v[t] += (v2[t] + (1LL << (-sh2 - 1))) >> (-sh2);
                    }
                }
                long long* dst = Crow + cb;
                if (!first && !last) {   // intermediate segment: reduce-add through L2, asynchronously
#pragma unroll
                    for (int h = 0; h < 2; ++h) {   // two halves of 8 values through the one slot
                        const int n = min(8, lim - 8 * h);
                        if (n <= 0) break;
                        if (nstg >= 1) bulk_wait_read_0();   // the slot's previous copy has been read
#pragma unroll
                        for (int t = 0; t < 8; t += 2)
                            if (t < n)
                                *reinterpret_cast<longlong2*>(stg + t * 8) = make_longlong2(v[8 * h + t], v[8 * h + t + 1]);
                        fence_proxy_async_shared();
                        bulk_reduce_add_s64(dst + 8 * h, smem_u32(stg), n * 8);
                        ++nstg;
                    }
                    continue;
                }
                if (!first) {   // add the accumulator (all loads first)
                    long long o[16];
                    if (v32) {
#pragma unroll
                        for (int t = 0; t < 16; t += 4) {
                            if (t < lim)
                                asm volatile("ld.global.v4.b64 {%0,%1,%2,%3}, [%4];"
                                             : "=l"(o[t]), "=l"(o[t + 1]), "=l"(o[t + 2]), "=l"(o[t + 3])
                                             : "l"(dst + t));
                            else
                                o[t] = o[t + 1] = o[t + 2] = o[t + 3] = 0;
                        }
                    } else {
#pragma unroll
                        for (int t = 0; t < 16; t += 2) {
                            if (t < lim) {
                                const longlong2 w = *reinterpret_cast<const longlong2*>(dst + t);
                                o[t] = w.x;
                                o[t + 1] = w.y;
                            } else {
                                o[t] = o[t + 1] = 0;
                            }
                        }
                    }
#pragma unroll
                    for (int t = 0; t < 16; ++t) v[t] += o[t];
                }
                if (last) {   // int64 fixed point -> FP64, in place
#pragma unroll
                    for (int t = 0; t < 16; t += 4) {
                        if (t >= lim) break;
                        const int4 eb4 = *reinterpret_cast<const int4*>(a.eB + cb + t);
                        const int ebv[4] = {eb4.x, eb4.y, eb4.z, eb4.w};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            double out;
                            if (ea == EXP_NAN || ebv[k] == EXP_NAN) {
                                out = __longlong_as_double(0x7ff8000000000000LL);
                            } else {
                                out = fixed_to_double(v[t + k], ea + ebv[k] + eoff + aexp);
                                out = __longlong_as_double(__double_as_longlong(out) ^ (long long)asign);
                                if (!apow2) out *= a.alpha;
                            }
                            v[t + k] = __double_as_longlong(out);
                        }
                    }
                }
                if (v32) {
#pragma unroll
                    for (int t = 0; t < 16; t += 4)
                        if (t < lim)
                            asm volatile("st.global.v4.b64 [%0], {%1,%2,%3,%4};" ::"l"(dst + t), "l"(v[t]),
                                         "l"(v[t + 1]), "l"(v[t + 2]), "l"(v[t + 3])
                                         : "memory");
                } else {
#pragma unroll
                    for (int t = 0; t < 16; t += 2)
                        if (t < lim) *reinterpret_cast<longlong2*>(dst + t) = make_longlong2(v[t], v[t + 1]);
                }
            }
            if (first && tot > 2) fence_proxy_async_global();   // plain stores before later reduce-adds
            tc_fence_before();
            mbar_arrive(&m.acce[b]);
            if (pair) mbar_arrive(&m.acce[b2]);
        }
        if (pair) break;   // group s-1 went with it
    }
    if (nstg) bulk_wait_all();   // staging reads done before the slots are reused or the CTA leaves
    if (total == 0 && row_ok) {   // every digit product of the tile is zero
        const int cbeg = c0 + half * (BN / 2);
        for (int c = cbeg; c < cbeg + BN / 2 && c < ncols; ++c) {
            const bool nan = ea == EXP_NAN || a.eB[c] == EXP_NAN;
            reinterpret_cast<double*>(Crow)[c] = nan ? __longlong_as_double(0x7ff8000000000000LL) : 0.0;
        }
    }
    return true;
}

// The launch's last CTA to finish zeroes the occupancy arrays the product read
// (every other CTA has finished reading them), for the splitter's next atomicMax
// accumulation, and resets the counter for the next launch.  A clear that does
// not happen (a launch cut short) leaves occupancy too high, never too low: more
// units are multiplied, and the result is the same.
__device__ __forceinline__ void clear_after_last(const SplitArgs& a) {
    if (!a.done) return;
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(a.done, 1u) == (unsigned int)a.nctas - 1u;
    }
    __syncthreads();
    if (!last) return;
    for (int i = threadIdx.x; i < a.clr_a_n; i += blockDim.x) a.clr_a[i] = 0;
    for (int i = threadIdx.x; i < a.clr_b_n; i += blockDim.x) a.clr_b[i] = 0;
    if (threadIdx.x == 0) *a.done = 0u;
}

// Teardown shared by both kernels.  By now the producer has settled its
// loads, the MMA thread its MMAs and every drain thread its bulk copies, so
// nothing is in flight: record an abort as a timeout, free TMEM and leave.
__device__ __forceinline__ void split_teardown(const SplitArgs& a, const SmemMap& m, uint32_t tmem, int warp) {
    __syncthreads();
    if (*m.abort_flag && threadIdx.x == 0) atomicExch(&a.st->timeout, 1);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

__device__ __forceinline__ void tmem_alloc_warp(const SmemMap& m) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(m.tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void init_barriers(const SmemMap& m) {
    for (int i = 0; i < STAGES; ++i) {
        mbar_init(&m.full[i], 1);
        mbar_init(&m.empty[i], 1);
    }
    for (int i = 0; i < NBUF; ++i) {
        mbar_init(&m.accf[i], 1);
        mbar_init(&m.acce[i], NDRAIN);
    }
    for (int i = 0; i < TSLOTS; ++i) {
        mbar_init(&m.tfull[i], 1);
        mbar_init(&m.tempty[i], NDRAIN);   // released by every drain thread after the tile's last drain
    }
    mbar_init(m.drain, 1);
    *m.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// ---------------------------------------------------------------------------
// One output tile per CTA (grouped launches, the allocation-free entry point,
// and no_persistent = 1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void zgemm_split_body(const CUtensorMap* tmA_p, const CUtensorMap* tmB_p,
                                                 const SplitArgs& a, int bid, bool global_maps) {
    if (zt_gate_skip(a.st, a.gate)) return;
    const SmemMap m = smem_map();
    TileSlot& ts = m.slots[0];
    int tig, tjg;
    if (!tile_group(a, bid, tig, tjg)) {   // the whole CTA leaves; it still counts as finished
        clear_after_last(a);
        return;
    }
    const int i0 = tig * BM, c0 = tjg * BN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = a.ldk / BK;

    if (threadIdx.x == 0) init_barriers(m);
    if (warp == 1) tmem_alloc_warp(m);
    if (warp == 2) fill_slot_warp(a, ts, tig, tjg, nkb, lane);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *m.tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            if (global_maps) {   // maps written by the host: visible to the tensormap proxy before use
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmA_p) : "memory");
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmB_p) : "memory");
            }
            int stage = 0;
            uint32_t ph = 0;
            long long nload = 0;
            produce_tile(a, ts, m, tmA_p, tmB_p, i0, c0, nkb, stage, ph, nload);
            producer_settle(m, nload);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0, seg = 0;
            uint32_t ph = 0;
            unsigned long long issued = 0;
            mma_tile(a, ts, m, tmem, nkb, stage, ph, seg, issued);
            mma_settle(m, a, issued);
        }
    } else if (warp < 2 + NDRAIN / 32) {
        int seg = 0;
        drain_tile(a, ts, m, tmem, i0, c0, warp, lane, seg);
    }
    split_teardown(a, m, tmem, warp);
    clear_after_last(a);
}

// ---------------------------------------------------------------------------
// Persistent form: one CTA per SM works through the launch order, taking
// tiles from a ticket counter (zeroed by the host before every launch).  A
// scheduler warp fills a ring of tile slots ahead of the roles, and the
// accumulator buffers rotate across tiles, so the last drain and the FP64
// epilogue of one tile overlap the first MMAs of the next.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void zgemm_split_persistent_body(const CUtensorMap* tmA_p, const CUtensorMap* tmB_p,
                                                            const SplitArgs& a) {
    if (zt_gate_skip(a.st, a.gate)) return;
    const SmemMap m = smem_map();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = a.ldk / BK;

    if (threadIdx.x == 0) init_barriers(m);
    if (warp == 1) tmem_alloc_warp(m);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *m.tmem_slot;

    if (warp == 0) {   // ---- TMA producer ----
        if (lane == 0) {
            int stage = 0;
            uint32_t ph = 0;
            long long nload = 0;
            for (int k = 0;; ++k) {
                const TileSlot& ts = m.slots[k % TSLOTS];
                if (!mbar_wait(&m.tfull[k % TSLOTS], (k / TSLOTS) & 1, m.abort_flag, a.wait_ns) || !ts.valid) break;
                if (!produce_tile(a, ts, m, tmA_p, tmB_p, ts.tig * BM, ts.tjg * BN, nkb, stage, ph, nload)) break;
            }
            producer_settle(m, nload);
        }
    } else if (warp == 1) {   // ---- MMA issuer ----
        if (lane == 0) {
            int stage = 0, seg = 0;
            uint32_t ph = 0;
            unsigned long long issued = 0;
            for (int k = 0;; ++k) {
                const TileSlot& ts = m.slots[k % TSLOTS];
                if (!mbar_wait(&m.tfull[k % TSLOTS], (k / TSLOTS) & 1, m.abort_flag, a.wait_ns) || !ts.valid) break;
                if (!mma_tile(a, ts, m, tmem, nkb, stage, ph, seg, issued)) break;
            }
            mma_settle(m, a, issued);
        }
    } else if (warp < 2 + NDRAIN / 32) {   // ---- drain / epilogue ----
        int seg = 0;
        for (int k = 0;; ++k) {
            const TileSlot& ts = m.slots[k % TSLOTS];
            if (!mbar_wait(&m.tfull[k % TSLOTS], (k / TSLOTS) & 1, m.abort_flag, a.wait_ns) || !ts.valid) break;
            if (!drain_tile(a, ts, m, tmem, ts.tig * BM, ts.tjg * BN, warp, lane, seg)) break;
            mbar_arrive(&m.tempty[k % TSLOTS]);   // this thread is done with the slot
        }
    } else {   // ---- scheduler: tile slots filled ahead of the roles ----
        for (int k = 0;; ++k) {
            TileSlot& ts = m.slots[k % TSLOTS];
            if (!mbar_wait(&m.tempty[k % TSLOTS], ((k / TSLOTS) & 1) ^ 1, m.abort_flag, a.wait_ns)) break;
            unsigned int ticket = 0;
            if (lane == 0) ticket = atomicAdd(a.tickets, 1u);
            ticket = __shfl_sync(0xffffffffu, ticket, 0);
            int tig = 0, tjg = 0;
            if (ticket >= (unsigned)a.ngroups || !tile_group(a, (int)ticket, tig, tjg)) {
                if (lane == 0) {
                    ts.valid = 0;
                    __threadfence_block();
                    mbar_arrive(&m.tfull[k % TSLOTS]);
                }
                break;
            }
            fill_slot_warp(a, ts, tig, tjg, nkb, lane);
            if (lane == 0) mbar_arrive(&m.tfull[k % TSLOTS]);
        }
    }
    split_teardown(a, m, tmem, warp);
    clear_after_last(a);
}

__global__ void __launch_bounds__(NTHREADS, CTAS_PER_SM)
zgemm_split_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const SplitArgs a) {
    zgemm_split_body(&tmA, &tmB, a, blockIdx.x, false);
}

__global__ void __launch_bounds__(NTHREADS, CTAS_PER_SM)
zgemm_split_persistent(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                       const SplitArgs a) {
    zgemm_split_persistent_body(&tmA, &tmB, a);
}

// Grouped: instances (each with its own tensor maps in global memory) share one launch.
__global__ void __launch_bounds__(NTHREADS, CTAS_PER_SM)
zgemm_split_grouped(const GemmEntry* tab, const int* offs, int n, int gate) {
    const int inst = zt_group_find(offs, n, blockIdx.x);
    const GemmEntry* e = tab + inst;
    SplitArgs a = e->a;
    a.gate = gate;
    zgemm_split_body(&e->tmA, &e->tmB, a, blockIdx.x - offs[inst], true);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

static int make_map(CUtensorMap* map, void* base, int rows, int ldk, int box_rows) {
    auto enc = encode_fn();
    if (!enc) return zt_fail(ZT_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ldk * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return zt_fail(ZT_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return ZT_OK;
}

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

int zt_split_create(zt_plan* p) {
    const int N = p->N;
    const int s = p->tun.slices, beta = p->tun.digit_bits, eg = p->tun.exact_groups;
    if (s < 3 || s > 8) return zt_fail(ZT_EINVAL, "slices=%d outside [3, 8]", s);
    if (beta < 6 || beta > 8) return zt_fail(ZT_EINVAL, "digit_bits=%d outside [6, 8]", beta);
    if (eg < 1 || eg > s) return zt_fail(ZT_EINVAL, "exact_groups=%d outside [1, slices]", eg);
    if (s * beta > 62) return zt_fail(ZT_EINVAL, "slices*digit_bits must be <= 62");
    if (p->tun.slices2 != 0 && (p->tun.slices2 < 2 || p->tun.slices2 > s))
        return zt_fail(ZT_EINVAL, "slices2=%d outside [2, slices]", p->tun.slices2);
    zt_split_ws* w = new (std::nothrow) zt_split_ws();
    if (!w) return zt_fail(ZT_ENOMEM, "host allocation failed");
    p->split = w;
    w->s = s;
    w->beta = beta;
    w->exact_groups = eg;
    w->wait_ns = (unsigned long long)p->tun.wait_us * 1000ull;
    w->stall_loads = p->tun.debug_stall_loads;
    w->skip_zero = p->tun.dense ? 0 : 1;
    w->ldk = round_up(2 * N, BK);
    w->Mpad = round_up(N, BM);
    w->Npad = round_up(2 * N, BN);
    // smallest u >= 0 with the worst-case int64 accumulator below 2^62 (for s and s2 digits)
    auto shift_for = [&](int sd) {
        const double R = std::ldexp(1.0, beta);
        double bound = 0.0;
        for (int g = 0; g < sd; ++g) bound += (g + 1) * std::pow(R, sd - 1 - g);
        bound *= (double)w->ldk * std::ldexp(1.0, 2 * beta - 2);
        int u = 0;
        while (bound >= std::ldexp(1.0, 62 + u)) ++u;
        return u;
    };
    w->u = shift_for(s);
    w->s2 = p->tun.slices2 ? p->tun.slices2 : s;
    w->u2 = shift_for(w->s2);
    cudaStream_t cs = p->mstream;   // the plan's private stream (synchronised at the end of plan creation)
    const size_t szA = (size_t)s * w->Mpad * w->ldk * sizeof(__nv_bfloat16);
    const size_t szB = (size_t)s * w->Npad * w->ldk * sizeof(__nv_bfloat16);
    ZT_CU(ZT_DMALLOC(w->dA, szA, cs));
    ZT_CU(cudaMemsetAsync(w->dA, 0, szA, cs));   // padding rows/columns stay zero
    ZT_CU(ZT_DMALLOC(w->eA, (size_t)w->Mpad * sizeof(int), cs));
    ZT_CU(cudaMemsetAsync(w->eA, 0, (size_t)w->Mpad * sizeof(int), cs));
    int rc;
    if ((rc = make_map(&w->tmA, w->dA, s * w->Mpad, w->ldk, BM))) return rc;
    w->nkb = w->ldk / BK;
    if (w->nkb > MAX_KB) return zt_fail(ZT_EINVAL, "N too large for the split product (K blocks > %d)", MAX_KB);
    w->ngA = w->Mpad / BM;
    w->ngB = w->Npad / BN;
    ZT_CU(ZT_DMALLOC(w->occA, (size_t)w->ngA * w->nkb * sizeof(int), cs));
    ZT_CU(cudaMemsetAsync(w->occA, 0, (size_t)w->ngA * w->nkb * sizeof(int), cs));
    for (int b = 0; b < 2; ++b) {
        ZT_CU(ZT_DMALLOC(w->occB[b], (size_t)w->ngB * w->nkb * sizeof(int), cs));
        ZT_CU(cudaMemsetAsync(w->occB[b], 0, (size_t)w->ngB * w->nkb * sizeof(int), cs));
        ZT_CU(ZT_DMALLOC(w->dB[b], szB, cs));
        ZT_CU(cudaMemsetAsync(w->dB[b], 0, szB, cs));
        ZT_CU(ZT_DMALLOC(w->eB[b], (size_t)w->Npad * sizeof(int), cs));
        ZT_CU(cudaMemsetAsync(w->eB[b], 0, (size_t)w->Npad * sizeof(int), cs));
        if ((rc = make_map(&w->tmB[b], w->dB[b], s * w->Npad, w->ldk, BN))) return rc;
    }
    // Launch orders.  0, 3, 4, 5: column blocks of 8, 16, 4 or 2 tiles, rows
    // walked inside a block, so that the tiles resident at one time share a
    // few B'^T panels across many rows (at N = 4096 the digit planes exceed
    // L2: DRAM reads per product fall from 8.0 to 5.0 GB against row-major
    // with blocks of 8; narrower blocks keep the active panels inside L2).
    // 1: row-major.  2: with all-zero digit tiles skipped, tiles near the
    // diagonal (where the leading digits of both operands are nonzero) carry
    // most of the work, so they are dispatched first and the light far tiles
    // fill the tail (longest-first ordering).  6: column blocks of 8 taken from
    // the last to the first: the first block ends with the tiles farthest from
    // the diagonal, so the light tiles fill the tail and the panels still share
    // L2 as in order 0.
    {
        const int ntmg = w->Mpad / BM, ntng = w->Npad / BN;
        const int order = p->tun.tile_order;
        const int cblk = (order == 0 || order == 6) ? 8 : order == 3 ? 16 : order == 4 ? 4 : order == 5 ? 2 : ntng;
        std::vector<std::pair<double, int>> full, lower;
        std::vector<int> blocks;
        for (int cb0 = 0; cb0 < ntng; cb0 += cblk) blocks.push_back(cb0);
        if (order == 6) std::reverse(blocks.begin(), blocks.end());
        for (int cb0 : blocks)
            for (int tg = 0; tg < ntmg; ++tg)
                for (int ug = cb0; ug < cb0 + cblk && ug < ntng; ++ug) {
                    const double dist = std::fabs((double)tg - (double)ug);
                    full.push_back({dist, tg * ntng + ug});
                    if (ug < tg + 1) lower.push_back({dist, tg * ntng + ug});
                }
        if (order == 2) {   // otherwise the enumeration order above
            std::stable_sort(full.begin(), full.end(), [](auto& x, auto& y) { return x.first < y.first; });
            std::stable_sort(lower.begin(), lower.end(), [](auto& x, auto& y) { return x.first < y.first; });
        }
        std::vector<int> of, ol;
        for (auto& e : full) of.push_back(e.second);
        for (auto& e : lower) ol.push_back(e.second);
        w->n_full = (int)of.size();
        w->n_lower = (int)ol.size();
        ZT_CU(ZT_DMALLOC(w->order_full, of.size() * sizeof(int), cs));
        ZT_CU(ZT_DMALLOC(w->order_lower, ol.size() * sizeof(int), cs));
        ZT_CU(cudaMemcpyAsync(w->order_full, of.data(), of.size() * sizeof(int), cudaMemcpyHostToDevice, cs));
        ZT_CU(cudaMemcpyAsync(w->order_lower, ol.data(), ol.size() * sizeof(int), cudaMemcpyHostToDevice, cs));
        ZT_CU(cudaStreamSynchronize(cs));   // host vectors go out of scope
    }
    w->persistent = p->tun.no_persistent ? 0 : 1;
    w->persistent2 = p->tun.second_form == 0 ? w->persistent : (p->tun.second_form == 2 ? 1 : 0);
    ZT_CU(cudaDeviceGetAttribute(&w->nsm, cudaDevAttrMultiProcessorCount, p->device));
    ZT_CU(ZT_DMALLOC(w->tickets, 16, cs));   // [0] tile tickets, [1] finished CTAs
    ZT_CU(cudaMemsetAsync(w->tickets, 0, 16, cs));
    if (zt_attr_needed(ZT_ATTR_SPLIT)) {
        ZT_CU(cudaFuncSetAttribute(zgemm_split_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
        ZT_CU(cudaFuncSetAttribute(zgemm_split_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)SMEM_BYTES));
        ZT_CU(cudaFuncSetAttribute(zgemm_split_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)SMEM_BYTES));
    }
    return ZT_OK;
}

size_t zt_split_bytes(int N, const zt_tuning& t) {
    const int s = t.slices;
    const size_t ldk = (size_t)round_up(2 * N, BK), Mpad = (size_t)round_up(N, BM),
                 Npad = (size_t)round_up(2 * N, BN);
    const size_t nkb = ldk / BK, ngA = Mpad / BM, ngB = Npad / BN;
    return (size_t)s * Mpad * ldk * 2 + 2 * (size_t)s * Npad * ldk * 2 + Mpad * 4 + 2 * Npad * 4 +
           ngA * nkb * 4 + 2 * ngB * nkb * 4 + 16;
}

void zt_split_destroy(zt_plan* p) {
    zt_split_ws* w = p->split;
    if (!w) return;
    cudaStream_t ms = p->mstream;
    zt_dfree(w->dA, ms);
    zt_dfree(w->eA, ms);
    zt_dfree(w->occA, ms);
    zt_dfree(w->order_full, ms);
    zt_dfree(w->order_lower, ms);
    zt_dfree(w->tickets, ms);
    for (int b = 0; b < 2; ++b) {
        zt_dfree(w->dB[b], ms);
        zt_dfree(w->eB[b], ms);
        zt_dfree(w->occB[b], ms);
    }
    delete w;
    p->split = nullptr;
}

int zt_split_rows_args(zt_plan* p, const double2* X, int to_a, int b_slot, SplitRowsArgs* out) {
    zt_split_ws* w = p->split;
    if (!w) return zt_fail(ZT_EINVAL, "plan has no split-precision workspace");
    SplitRowsArgs& a = *out;
    // B'^T slot 1 holds s2 digits; a split into X' and slot 1 at once needs s2 == s
    if (b_slot == 1 && to_a && w->s2 != w->s)
        return zt_fail(ZT_EINVAL, "split into X' and slot 1 at once needs slices2 == slices");
    a.X = X;
    a.N = p->N;
    a.s = b_slot == 1 ? w->s2 : w->s;
    a.beta = w->beta;
    a.ldk = w->ldk;
    a.dA = to_a ? w->dA : nullptr;
    a.Mpad = w->Mpad;
    a.eA = to_a ? w->eA : nullptr;
    a.dB = b_slot >= 0 ? w->dB[b_slot] : nullptr;
    a.Npad = w->Npad;
    a.eB = b_slot >= 0 ? w->eB[b_slot] : nullptr;
    a.occA = to_a ? w->occA : nullptr;
    a.occA_rows = BM;
    a.occA_n = w->ngA * w->nkb;
    a.occB = b_slot >= 0 ? w->occB[b_slot] : nullptr;
    a.occB_rows = BN / 2;
    a.occB_n = w->ngB * w->nkb;
    a.st = p->state;
    a.gate = ZT_GATE_NONE;
    return ZT_OK;
}

int zt_split_rows_grouped(const SplitRowsArgs* tab, const int* offs, int n, int total, cudaStream_t s, int gate) {
    // occupancy arrays start at zero: the products that read them clear them
    split_rows_grouped<<<total, 256, 0, s>>>(tab, offs, n, gate);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "split_rows_grouped");
    return ZT_OK;
}

int zt_split_operand(zt_plan* p, const double2* X, int to_a, int b_slot, cudaStream_t s, int gate) {
    zt_split_ws* w = p->split;
    if (!w) return zt_fail(ZT_EINVAL, "plan has no split-precision workspace");
    const int N = p->N;
    SplitRowsArgs ra;
    int rc = zt_split_rows_args(p, X, to_a, b_slot, &ra);
    if (rc) return rc;
    ra.gate = gate;
    const double bytes = 16.0 * N * N + (to_a ? 2.0 * w->s * (double)N * w->ldk : 0.0) +
                         (b_slot >= 0 ? 4.0 * w->s * (double)N * w->ldk : 0.0);
    // occupancy is reduced with atomicMax over the rows of each group; the arrays are
    // zero here (plan creation, then cleared by the product that read them)
    const int t = zt_timer_begin(p, ZT_KERNEL_SPLIT, bytes, bytes, s);
    split_rows_kernel<<<N, 256, 0, s>>>(ra);
    zt_timer_end(p, t, s);
    p->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "split_rows_kernel");
    return ZT_OK;
}

__global__ void __launch_bounds__(256) split_rows2_kernel(const SplitRowsArgs a0, const SplitRowsArgs a1, int n0) {
    if ((int)blockIdx.x < n0)
        split_rows_body(a0, blockIdx.x);
    else
        split_rows_body(a1, blockIdx.x - n0);
}

int zt_split_operands2(zt_plan* p, const double2* X1, const double2* X2, cudaStream_t s, int gate) {
    zt_split_ws* w = p->split;
    if (!w) return zt_fail(ZT_EINVAL, "plan has no split-precision workspace");
    const int N = p->N;
    SplitRowsArgs r1, r2;
    int rc;
    if ((rc = zt_split_rows_args(p, X1, 1, -1, &r1)) || (rc = zt_split_rows_args(p, X2, 0, 0, &r2))) return rc;
    r1.gate = r2.gate = gate;
    const double bytes = 2 * 16.0 * N * N + 2.0 * w->s * (double)N * w->ldk + 4.0 * w->s * (double)N * w->ldk;
    const int t = zt_timer_begin(p, ZT_KERNEL_SPLIT, bytes, bytes, s);
    split_rows2_kernel<<<2 * N, 256, 0, s>>>(r1, r2, N);
    zt_timer_end(p, t, s);
    p->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "split_rows2_kernel");
    return ZT_OK;
}

static void product_args(zt_plan* p, int b_slot, double2* C, double alpha, int lower_only, int keep_a,
                         SplitArgs& a, int* ngroups_out) {
    zt_split_ws* w = p->split;
    const int N = p->N;
    a.N = N;
    // a product with slot 1 takes s2 digit groups: the leading s2 planes of X' (a
    // plane's weight does not depend on how many planes follow it) and slot 1's s2
    a.s = b_slot == 1 ? w->s2 : w->s;
    a.s_occA = w->s;
    a.beta = w->beta;
    a.ldk = w->ldk;
    a.Mpad = w->Mpad;
    a.Npad = w->Npad;
    a.u = b_slot == 1 ? w->u2 : w->u;
    a.exact_groups = w->exact_groups;
    a.ntn = w->Npad / BN;
    a.lower_only = lower_only;
    a.ntng = w->Npad / BN;
    a.wait_ns = w->wait_ns;
    a.stall_loads = w->stall_loads;
    a.occA = w->skip_zero ? w->occA : nullptr;
    a.occB = w->skip_zero ? w->occB[b_slot] : nullptr;
    a.units = nullptr;
    a.alpha = alpha;
    a.eA = w->eA;
    a.eB = w->eB[b_slot];
    a.C = reinterpret_cast<double*>(C);
    a.st = p->state;
    a.gate = ZT_GATE_NONE;
    a.order = lower_only ? w->order_lower : w->order_full;   // only tiles with work
    const int ngroups = lower_only ? w->n_lower : w->n_full;
    a.ngroups = ngroups;
    a.tickets = nullptr;
    if (w->skip_zero) {   // the occupancy this product reads is cleared by its last CTA
        a.clr_a = keep_a ? nullptr : w->occA;   // keep_a: the X' planes serve a later product too
        a.clr_a_n = keep_a ? 0 : w->ngA * w->nkb;
        a.clr_b = w->occB[b_slot];
        a.clr_b_n = w->ngB * w->nkb;
        a.done = w->tickets + 1;
    } else {
        a.clr_a = a.clr_b = nullptr;
        a.clr_a_n = a.clr_b_n = 0;
        a.done = nullptr;
    }
    a.nctas = ngroups;   // one tile per CTA; the persistent launch sets its grid
    *ngroups_out = ngroups;
}

int zt_split_gemm_entry(zt_plan* p, int b_slot, double2* C, double alpha, int lower_only, int keep_a,
                        GemmEntry* out, int* ctas) {
    zt_split_ws* w = p->split;
    if (!w) return zt_fail(ZT_EINVAL, "plan has no split-precision workspace");
    int ngroups;
    product_args(p, b_slot, C, alpha, lower_only, keep_a, out->a, &ngroups);
    out->tmA = w->tmA;
    out->tmB = w->tmB[b_slot];
    *ctas = ngroups;
    return ZT_OK;
}

int zt_split_gemm_grouped(const GemmEntry* tab, const int* offs, int n, int total, cudaStream_t s, int gate) {
    zgemm_split_grouped<<<total, NTHREADS, SMEM_BYTES, s>>>(tab, offs, n, gate);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "zgemm_split_grouped");
    return ZT_OK;
}

int zt_split_product(zt_plan* p, int b_slot, double2* C, double alpha, int lower_only, int keep_a, cudaStream_t s,
                     int gate) {
    zt_split_ws* w = p->split;
    if (!w) return zt_fail(ZT_EINVAL, "plan has no split-precision workspace");
    const int N = p->N;
    SplitArgs a;
    int ngroups;
    product_args(p, b_slot, C, alpha, lower_only, keep_a, a, &ngroups);
    a.gate = gate;
    a.units = p->timing ? p->d_units : nullptr;   // issued work is counted on the device
    const double alg = lower_only ? 4.0 * N * (double)N * (N + 1.0) : 8.0 * (double)N * N * N;
    const int t = zt_timer_begin(p, ZT_KERNEL_PRODUCT, 0.0, alg, s);
    cudaError_t e;
    if (b_slot == 1 ? w->persistent2 : w->persistent) {   // one CTA per SM works through the tile groups
        e = cudaMemsetAsync(w->tickets, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) {
            zt_timer_end(p, t, s);
            return zt_cuda_check(e, "cudaMemsetAsync(tickets)");
        }
        a.tickets = w->tickets;
        const int grid = ngroups < w->nsm ? ngroups : w->nsm;
        a.nctas = grid;
        if (grid > 0) zgemm_split_persistent<<<grid, NTHREADS, SMEM_BYTES, s>>>(w->tmA, w->tmB[b_slot], a);
    } else {
        zgemm_split_kernel<<<ngroups, NTHREADS, SMEM_BYTES, s>>>(w->tmA, w->tmB[b_slot], a);
    }
    zt_timer_end(p, t, s);
    p->launches++;
    e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "zgemm_split_kernel");
    return ZT_OK;
}

int zt_launch_zgemm_split(zt_plan* p, const double2* X, const double2* Y, double2* C, double alpha,
                          int lower_only, cudaStream_t s, int gate) {
    int rc;
    if ((rc = zt_split_operand(p, X, 1, -1, s, gate))) return rc;
    if ((rc = zt_split_operand(p, Y, 0, 0, s, gate))) return rc;
    return zt_split_product(p, 0, C, alpha, lower_only, 0, s, gate);
}

// ---------------------------------------------------------------------------
// Allocation-free split-precision product (no counterpart in the paper).
//
// For callers that cannot allocate device memory, the scratch of the split
// product (digit planes of X' and B'^T, row exponents, a status word) lives
// in one file-scope device array sized for N <= ZT_NOALLOC_MAX_N, laid out
// once for that maximum (Mpad = 256 rows, Npad = 512 rows, K' = 512).  The
// host never dereferences the array's name: its device address is resolved
// per device with cudaGetSymbolAddress on first use and passed to the
// kernels.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {
constexpr int NA_S = 7, NA_BETA = 7, NA_EG = 4;
constexpr int NA_MPAD = 256, NA_NPAD = 512, NA_LDK = 512;
constexpr size_t NA_DA = (size_t)NA_S * NA_MPAD * NA_LDK * 2;
constexpr size_t NA_DB = (size_t)NA_S * NA_NPAD * NA_LDK * 2;
constexpr size_t NA_EA = (size_t)NA_MPAD * sizeof(int);
constexpr size_t NA_EB = (size_t)NA_NPAD * sizeof(int);
constexpr size_t NA_ST = 256;
constexpr size_t NA_BYTES = NA_DA + NA_DB + NA_EA + NA_EB + NA_ST;
static_assert(NA_BYTES == ZT_NOALLOC_SCRATCH_BYTES, "scratch size must match the header");
static_assert(2 * ZT_NOALLOC_MAX_N <= NA_LDK && ZT_NOALLOC_MAX_N <= NA_MPAD && 2 * ZT_NOALLOC_MAX_N <= NA_NPAD,
              "scratch layout too small for ZT_NOALLOC_MAX_N");
static_assert(sizeof(zt_dev_state) <= NA_ST, "status word does not fit");
constexpr int NA_MAX_DEVICES = 64;

struct NoAllocDevice {
    bool ready = false;
    unsigned char* base = nullptr;   // device address of zt_noalloc_scratch on this device
};
NoAllocDevice g_noalloc[NA_MAX_DEVICES];
std::mutex g_noalloc_mu;
}  // namespace

static __device__ __align__(256) unsigned char zt_noalloc_scratch[NA_BYTES];

// Once per device, with that device current: resolve the array's device
// address and raise the product kernel's dynamic shared-memory limit.
static int noalloc_setup(unsigned char** base) {
    int dev = -1;
    ZT_CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return zt_fail(ZT_EINVAL, "device ordinal %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc[dev].ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, zt_noalloc_scratch);
        if (e != cudaSuccess) return zt_cuda_check(e, "cudaGetSymbolAddress(zt_noalloc_scratch)");
        e = cudaFuncSetAttribute(zgemm_split_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        if (e != cudaSuccess) return zt_cuda_check(e, "cudaFuncSetAttribute(zgemm_split_kernel)");
        g_noalloc[dev].base = static_cast<unsigned char*>(p);
        g_noalloc[dev].ready = true;
    }
    *base = g_noalloc[dev].base;
    return ZT_OK;
}

extern "C" int zt_zgemm_skew_split_noalloc(int N, const double* X, const double* Y, double* C, void* stream) {
    if (N < 1 || N > ZT_NOALLOC_MAX_N)
        return zt_fail(ZT_EINVAL, "zt_zgemm_skew_split_noalloc: N=%d outside [1, %d] (static scratch limit)", N,
                       ZT_NOALLOC_MAX_N);
    if (!X || !Y || !C) return zt_fail(ZT_EINVAL, "zt_zgemm_skew_split_noalloc: NULL matrix");
    if ((((uintptr_t)X) | ((uintptr_t)Y) | ((uintptr_t)C)) & 15u)
        return zt_fail(ZT_EINVAL, "zt_zgemm_skew_split_noalloc: matrices must be 16-byte aligned");
    if (C == X || C == Y) return zt_fail(ZT_EINVAL, "zt_zgemm_skew_split_noalloc: C must not alias X or Y");
    unsigned char* base = nullptr;
    int rc = noalloc_setup(&base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    __nv_bfloat16* dA = reinterpret_cast<__nv_bfloat16*>(base);
    __nv_bfloat16* dB = reinterpret_cast<__nv_bfloat16*>(base + NA_DA);
    int* eA = reinterpret_cast<int*>(base + NA_DA + NA_DB);
    int* eB = reinterpret_cast<int*>(base + NA_DA + NA_DB + NA_EA);
    zt_dev_state* st = reinterpret_cast<zt_dev_state*>(base + NA_DA + NA_DB + NA_EA + NA_EB);
    // The array keeps the previous call's contents: padding rows and columns
    // of the digit planes and the status word must start at zero.
    ZT_CU(cudaMemsetAsync(base, 0, NA_BYTES, s));
    CUtensorMap tmA, tmB;
    if ((rc = make_map(&tmA, dA, NA_S * NA_MPAD, NA_LDK, BM))) return rc;
    if ((rc = make_map(&tmB, dB, NA_S * NA_NPAD, NA_LDK, BN))) return rc;
    int u = 0;
    {
        const double R = std::ldexp(1.0, NA_BETA);
        double bound = 0.0;
        for (int g = 0; g < NA_S; ++g) bound += (g + 1) * std::pow(R, NA_S - 1 - g);
        bound *= (double)NA_LDK * std::ldexp(1.0, 2 * NA_BETA - 2);
        while (bound >= std::ldexp(1.0, 62 + u)) ++u;
    }
    SplitRowsArgs ra = {};
    ra.X = (const double2*)X;
    ra.N = N;
    ra.s = NA_S;
    ra.beta = NA_BETA;
    ra.ldk = NA_LDK;
    ra.dA = dA;
    ra.Mpad = NA_MPAD;
    ra.eA = eA;
    ra.Npad = NA_NPAD;
    ra.occA_rows = ra.occB_rows = 1;   // no occupancy tracking (every digit pair is multiplied)
    ra.st = st;
    ra.gate = ZT_GATE_NONE;
    split_rows_kernel<<<N, 256, 0, s>>>(ra);
    ra.X = (const double2*)Y;
    ra.dA = nullptr;
    ra.eA = nullptr;
    ra.dB = dB;
    ra.eB = eB;
    split_rows_kernel<<<N, 256, 0, s>>>(ra);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "split_rows_kernel");
    SplitArgs a;
    a.N = N;
    a.s = NA_S;
    a.s_occA = NA_S;
    a.beta = NA_BETA;
    a.ldk = NA_LDK;
    a.Mpad = NA_MPAD;
    a.Npad = NA_NPAD;
    a.u = u;
    a.exact_groups = NA_EG;
    a.ntn = NA_NPAD / BN;
    a.lower_only = 0;
    a.tickets = nullptr;
    a.ntng = NA_NPAD / BN;
    a.wait_ns = 2000000000ull;
    a.stall_loads = 0;
    a.clr_a = a.clr_b = nullptr;
    a.clr_a_n = a.clr_b_n = 0;
    a.done = nullptr;
    a.nctas = 0;
    a.occA = nullptr;   // no zero-unit skipping: every digit pair is multiplied
    a.occB = nullptr;
    a.units = nullptr;
    a.order = nullptr;
    a.ngroups = (NA_MPAD / BM) * (NA_NPAD / BN);
    a.alpha = -1.0;
    a.eA = eA;
    a.eB = eB;
    a.C = C;
    a.st = st;
    a.gate = ZT_GATE_NONE;
    zgemm_split_kernel<<<(NA_MPAD / BM) * (NA_NPAD / BN), NTHREADS, SMEM_BYTES, s>>>(tmA, tmB, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return zt_cuda_check(e, "zgemm_split_kernel");
    zt_dev_state hs;
    ZT_CU(cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s));
    ZT_CU(cudaStreamSynchronize(s));
    if (hs.timeout) return zt_fail(ZT_ETIMEOUT, "zt_zgemm_skew_split_noalloc: bounded device wait ran out");
    return ZT_OK;
}
