// Kinetic-energy spectrum E_l (Sec. 4) over the quantised basis (Sec. 3.2).
//
// E_l = sum_{|m| <= l} |omega_lm|^2 / (2 l (l+1)), l >= 1, E_0 = 0, where
// |omega_{l,+-m}| = |v^T w_{+-m}| / |v| for the eigenvector v of the block
// -Delta^m (Eq. 13) at the eigenvalue l(l+1) (Eq. 12), and w_{+-m} are the
// diagonals +-m of W (lower: W[i+m, i], upper: W[i, i+m]).  For W in su(N)
// the upper diagonal is -conj of the lower, so |omega_{l,-m}| = |omega_lm|
// and only the lower triangle is read.  The E_l sum to the Hamiltonian
// (1/2) tr(P W), P = Delta_N^{-1} W.
//
// Every eigenvector of every block takes part (N^3/3 work) and none is stored.
//
// Factorisation.  On diagonal m, -Delta = ad(S-) ad(S+) + m(m+1) (the spin
// Casimir behind Hoppe's Laplacian), so -Delta^m = C^T C + m(m+1) I with C the
// bidiagonal map ad(S+) from diagonal m to m + 1:
//     (C x)_i = p_i x_i + q_i x_{i+1},  p_i = sqrt((i+m+1)(N-1-i-m)),
//                                       q_i = -sqrt((i+1)(N-1-i)),
// (a_i = p_i^2 + q_{i-1}^2 + m(m+1), b_i = p_i q_i: the entries of Eq. 13).
// At l(l+1) the shifted eigenvalue mu = (l-m)(l+m+1) is an exact integer and
// the eigenvector x follows from C x = g, C^T g = mu x read row by row:
//     g_i     = (mu x_i - q_{i-1} g_{i-1}) / p_i,
//     x_{i+1} = (g_i - p_i x_i) / q_i,           x_0 = 1, g_{-1} = 0,
// carried as G_i = g_i / q_i (4 FP64 instructions per step):
//     G_i     = (mu x_i - Q_i G_{i-1}) d_i,   Q_i = q_{i-1}^2 = i (N - i) exact,
//     x_{i+1} = G_i - r_i x_i,                 d_i = 1 / (p_i q_i), r_i = p_i / q_i.
// No step subtracts quantities of size N^2 to leave one of size l(l+1), as
// the three-term recurrence of the tridiagonal rows would (its low-l
// eigenvectors lose accuracy like N^2 eps); these factors fix the small
// eigenvalues to high relative accuracy.
//
// Half vectors.  The blocks are persymmetric, so x is even or odd about the
// centre of its diagonal, with parity (-1)^(l-m) (the reflection symmetry of
// the 3j symbols of Eq. 11).  The recurrence runs from the end of the
// diagonal to its centre only: the oscillatory range of the eigenvector is a
// central interval, and outside it the recurrence runs in the growing
// direction.  Folded diagonals w_i +- w_{n-1-i} turn the full dot product
// into one over the half.  x and G are rescaled by 2^-400 whenever |x|
// passes 2^400 (the end entries can be far below the double range relative
// to the bulk).
//
// One thread per (l, m): a CTA holds 128 consecutive l of one m and stages
// Q_i, d_i, r_i and the folded diagonal in shared memory, 128
// positions at a time, so the inner loop is FP64 FMAs on broadcast
// shared-memory operands with no division.  Per-(l, m) energies go to a
// packed triangle in the plan's workspace; a second kernel sums them over m
// in a fixed order.
#include "zt_internal.h"

namespace {
constexpr int SP_TH = 128;   // l values per CTA = positions staged per chunk
constexpr int SS_TH = 256;
}  // namespace

__global__ void __launch_bounds__(SP_TH) spectrum_pairs_kernel(const double2* __restrict__ W, int N,
                                                               double* __restrict__ e) {
    const int m = blockIdx.y, n = N - m;
    const int l0 = m + (int)blockIdx.x * SP_TH;
    if (l0 > N - 1) return;   // the whole CTA lies past the block
    const int tid = threadIdx.x;
    const int l = l0 + tid;
    const bool active = l <= N - 1;
    const int half = (n + 1) >> 1;
    const int par = (l - m) & 1;   // 0: even about the centre, 1: odd
    __shared__ double s_Q[SP_TH], s_d[SP_TH], s_r[SP_TH];
    __shared__ double2 s_f[2][SP_TH];   // folded lower diagonal: even, odd
    const double mu = (double)(l - m) * (double)(l + m + 1);
    double x = 1.0, G = 0.0, nrm = 0.0;
    double lr = 0.0, li = 0.0;
    for (int i0 = 0; i0 < half; i0 += SP_TH) {
        __syncthreads();   // the previous chunk is consumed
        const int i = i0 + tid;
        if (i < half) {
            // p_i, q_i are nonzero for i <= half - 2 < n - 1 (only those steps run)
            const double pv = sqrt((double)(i + m + 1) * (double)(N - 1 - i - m));
            const double qv = -sqrt((double)(i + 1) * (double)(N - 1 - i));
            s_Q[tid] = (double)i * (double)(N - i);
            s_d[tid] = (pv != 0.0 && qv != 0.0) ? 1.0 / (pv * qv) : 0.0;
            s_r[tid] = (qv != 0.0) ? pv / qv : 0.0;
            const int j = n - 1 - i;
            const double2 lo_i = W[(size_t)(i + m) * N + i];
            if (i == j) {   // centre of an odd-length diagonal: counted once, zero in odd vectors
                s_f[0][tid] = lo_i;
                s_f[1][tid] = make_double2(0.0, 0.0);
            } else {
                const double2 lo_j = W[(size_t)(j + m) * N + j];
                s_f[0][tid] = make_double2(lo_i.x + lo_j.x, lo_i.y + lo_j.y);
                s_f[1][tid] = make_double2(lo_i.x - lo_j.x, lo_i.y - lo_j.y);
            }
        }
        __syncthreads();
        if (active) {
            const int cnt = min(SP_TH, half - i0);
            const double2* fl = s_f[par];
            for (int k = 0; k < cnt; ++k) {
                const double2 wl = fl[k];
                lr = fma(x, wl.x, lr);
                li = fma(x, wl.y, li);
                nrm = fma(x, x, nrm);
                if (i0 + k + 1 < half) {
                    G = fma(-s_Q[k], G, mu * x) * s_d[k];
                    const double xn = fma(-s_r[k], x, G);
                    x = xn;
                    if ((__double2hiint(xn) & 0x7ff00000) > ((1023 + 400) << 20)) {
                        x *= 0x1p-400;
                        G *= 0x1p-400;
                        lr *= 0x1p-400;
                        li *= 0x1p-400;
                        nrm *= 0x1p-800;
                    }
                }
            }
        }
    }
    if (!active) return;
    // full norm: twice the half, the centre of an odd-length diagonal once
    // (x holds the last entry of the half, the centre when n is odd)
    double full = 2.0 * nrm;
    if (n & 1) full -= (par ? 2.0 : 1.0) * x * x;
    double num = lr * lr + li * li;
    if (m > 0) num *= 2.0;   // omega_{l,-m}: the mirrored upper diagonal (diagonal 0 is its own)
    e[zt_tri(l, m)] = num / full;
}

__global__ void __launch_bounds__(SS_TH) spectrum_sum_kernel(const double* __restrict__ e, int N,
                                                             double* __restrict__ E) {
    const int l = blockIdx.x * SS_TH + threadIdx.x;
    if (l >= N) return;
    double s = 0.0;
    const double* row = e + zt_tri(l, 0);
    for (int m = 0; m <= l; ++m) s += row[m];   // fixed order over m
    E[l] = (l > 0) ? s / (2.0 * (double)l * (double)(l + 1)) : 0.0;
}

extern "C" int zeitlin_energy_spectrum(zt_plan* p, const double* W, double* E, void* stream) {
    if (!p) return zt_fail(ZT_EINVAL, "plan is NULL");
    if (!W || (((uintptr_t)W) & 15u)) return zt_fail(ZT_EINVAL, "W is NULL or not 16-byte aligned");
    if (!E || (((uintptr_t)E) & 7u)) return zt_fail(ZT_EINVAL, "E is NULL or not 8-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const int N = p->N;
    double* e = reinterpret_cast<double*>(p->A);   // N(N+1)/2 doubles <= 2 N^2
    const dim3 grid((unsigned)((N + SP_TH - 1) / SP_TH), (unsigned)N);
    spectrum_pairs_kernel<<<grid, SP_TH, 0, s>>>((const double2*)W, N, e);
    spectrum_sum_kernel<<<(N + SS_TH - 1) / SS_TH, SS_TH, 0, s>>>(e, N, E);
    p->launches += 2;
    ZT_CU(cudaGetLastError());
    zt_note_use(p, s);
    return ZT_OK;
}
