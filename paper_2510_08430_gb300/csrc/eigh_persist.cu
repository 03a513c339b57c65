// Persistent, grid-synchronised kernels of the per-block solver (Sec. 2, block-layer
// paragraph; S~_b = S_b + lambda I, dtheta_b = -eta pinv(S~_b) F_b):
//
//  trd_persist_kernel    Householder reduction Q^H S_b Q = T of every block, all columns
//                        in one launch. Three phases per column j, separated by grid
//                        barriers:
//                          R  column j finalised (the alpha part of reflector j-1's update,
//                             b - 2 Re(alpha) v), its sub-diagonal norm, reflector j and v_j
//                             (stored in the upper part of row j), w_{j-1} = x_{j-1} + alpha v_{j-1};
//                          C  trailing lower triangle: pending rank-2 update of reflector j-1
//                             fused with the Hermitian matvec y = A v_j (64 x 64 tiles);
//                          X  x_j = tau_j y, column j+1 updated by reflector j except for its
//                             alpha part (b = a - v conj(x_{j+1}) - x), and the partials of
//                             x_j^H v_j that give alpha_j.
//  refine_persist_kernel Iterative refinement of the mixed-precision solve, all sweeps in
//                        one launch: x += Q (T + lambda I)^{-1} Q^H r with Q applied in
//                        blocked (WY) form, one panel of QNB reflectors per phase, then the
//                        FP64 residual r = F - (S + lambda I) x and the convergence test.
//
// All CTAs of a cooperative launch are co-resident. Work of a phase is split into units
// (row chunks or tiles of every active block) taken grid-stride. Data written in one
// phase and read in a later one use plain global loads, never the read-only path.
#include "eigh.cuh"

namespace nqs {
namespace {

constexpr int PT = 256;                              // threads per CTA (== CH)

static_assert(PT == CH, "one thread per row of a chunk");
static_assert(MAXB <= PT, "unit prefix holds one block per thread");

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier over all CTAs of the launch: bar[0] counts arrivals, bar[1] is the
// generation. The last arriver resets the count and advances the generation. A wait
// that exceeds `budget` ns records NQS_ERR_TIMEOUT and returns false; the caller returns.
__device__ bool grid_sync(unsigned* bar, DevStatus* status, int where, int* ok_s, unsigned long long budget) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = now_ns();
            while (*gen == g) {
                __nanosleep(64);
                if (now_ns() - t0 > budget) {
                    ok = 0;
                    set_status(status, NQS_ERR_TIMEOUT, where, -1);
                    break;
                }
            }
        }
        __threadfence();
        *ok_s = ok;
    }
    __syncthreads();
    return *ok_s != 0;
}

// pref[0..nb]: prefix of per-block unit counts (cnt(b) = 0 for a block idle in this
// phase). Called by all threads of the CTA; returns the total.
template <typename F>
__device__ long long unit_prefix(int nb, F cnt, long long* pref, long long* wsum) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    long long v = (t < nb) ? cnt(t) : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    __syncthreads();
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    long long add = 0;
    for (int k = 0; k < w; ++k) add += wsum[k];
    if (t < nb) pref[t + 1] = v + add;
    if (t == 0) pref[0] = 0;
    __syncthreads();
    return pref[nb];
}

// Block of unit u: the last b with pref[b] <= u (its count is then non-zero).
__device__ __forceinline__ int unit_block(const long long* pref, int nb, long long u) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pref[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int tri_index(long long t, int* I, int* J) {
    long long ii = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
    while (ii * (ii + 1) / 2 > t) --ii;
    *I = (int)ii;
    *J = (int)(t - ii * (ii + 1) / 2);
    return 0;
}

// ------------------------------------------------------------------ reduction phases
template <typename R> struct TrdSmem {
    cx<R> sv[2][TB], svp[2][TB], swp[2][TB];
    cx<R> p2buf[16][TB + 1];
    cx<R> p1s[TB];
};

// Between phase X of column j-1 and phase R of column j:
//   bcol[r]  = column j (rows [j, n)) updated by reflector j-1 except for its alpha part,
//              b = a - v_{j-1} conj(x_{j-1}[j]) - x_{j-1}; the full update is b - 2 Re(alpha) v;
//   pxv[u]   = sum conj(x_r) v_r over DCH-row unit u of rows [j, n) (gives alpha_{j-1}).

// Prologue: column 0 has nothing pending (b = a, x = v = 0). CTA unit c covers rows
// [c CH, c CH + CH); warp w clears DCH-unit c (CH/DCH) + w.
template <typename R>
__device__ void trd_prologue(const TrdBufs<R>& B, int b, int c) {
    const EBlk blk = B.tab[b];
    const int n = blk.n;
    const long long r = (long long)c * CH + threadIdx.x;
    if (r < n) B.bcol[blk.off + r] = B.A[blk.soff + r * n];
    if ((threadIdx.x & 31) == 0)
        B.pxv[(long long)b * MAXDCH + (long long)c * (CH / DCH) + (threadIdx.x >> 5)] = mk<double>(0.0, 0.0);
}

// R: column j on rows [j, n), chunk c (CH rows): finalise it, form reflector j
// (LAPACK-style: beta real, H^H [alpha; x] = [beta; 0]) and v_j, and w_{j-1}. Every unit
// computes the sub-diagonal norm of the final column itself (one pass over bcol).
template <typename R>
__device__ void trd_phase_r(const TrdBufs<R>& B, int b, int j, int c, const cx<R>* vprev, cx<R>* vcur, double* shd,
                            c128* shc, DevStatus* status) {
    const EBlk blk = B.tab[b];
    const int n = blk.n;
    cx<R>* A = B.A + blk.soff;
    const cx<R>* bc = B.bcol + blk.off;
    const cx<R>* vp = vprev + blk.off;
    if (threadIdx.x < 32) {
        const int K = (n - j + DCH - 1) / DCH;  // units of rows [j, n) of the previous phase
        c128 p1 = mk<double>(0.0, 0.0);
        for (int k = threadIdx.x; k < K; k += 32) p1 = p1 + B.pxv[(long long)b * MAXDCH + k];
        p1 = warp_sum(p1);
        if (threadIdx.x == 0) {
            const c128 alpha = j >= 1 ? (-0.5) * (B.tau[blk.off + j - 1] * p1) : mk<double>(0.0, 0.0);
            shc[0] = alpha;
        }
    }
    __syncthreads();
    const c128 alpha = shc[0];
    const R cc = (R)(2.0 * alpha.re);
    const bool pend = j >= 1;
    double xn = 0.0;
    for (int r = j + 2 + threadIdx.x; r < n; r += PT) {
        const cx<R> a = pend ? bc[r] - cc * vp[r] : bc[r];
        xn += cabs2(ccast<double>(a));  // squares in FP64: FP32 squares of tiny entries go subnormal
    }
    xn = block_sum(xn, shd);
    if (threadIdx.x == 0 && j <= n - 2) {
        const c128 al = ccast<double>(pend ? bc[j + 1] - cc * vp[j + 1] : bc[j + 1]);
        double beta;
        c128 tau, scale;
        if (xn == 0.0 && al.im == 0.0) {
            beta = al.re;
            tau = mk<double>(0.0, 0.0);
            scale = mk<double>(0.0, 0.0);
        } else {
            const double nrm = sqrt(al.re * al.re + al.im * al.im + xn);
            beta = (al.re >= 0.0) ? -nrm : nrm;
            tau = mk<double>((beta - al.re) / beta, -al.im / beta);
            const c128 dnm = mk<double>(al.re - beta, al.im);
            const double q = cabs2(dnm);
            scale = mk<double>(dnm.re / q, -dnm.im / q);
        }
        shc[1] = scale;
        if (c == 0) {
            if (!isfinite(beta) || !finite_cx(tau) || !finite_cx(scale))
                set_status(status, NQS_ERR_NONFINITE, W_TRD, (long long)blk.orig * 1000000 + j);
            B.e[blk.off + j] = beta;
            B.e2[blk.off + j] = beta * beta;
            B.tau[blk.off + j] = tau;
        }
    }
    __syncthreads();
    const long long r = (long long)j + (long long)c * CH + threadIdx.x;
    c128 vf = mk<double>(0.0, 0.0);
    if (r < n) {
        cx<R> a = bc[r];
        if (pend) {
            const cx<R> vr = vp[r];
            a = a - cc * vr;
            B.w[blk.off + r] = ccast<R>(ccast<double>(B.x[blk.off + r]) + alpha * ccast<double>(vr));
        }
        if (r == j) {
            B.d[blk.off + j] = (double)a.re;
        } else if (j <= n - 2) {
            const cx<R> v = (r == j + 1) ? mk<R>(R(1), R(0)) : a * ccast<R>(shc[1]);
            vcur[blk.off + r] = v;
            A[(long long)j * n + r] = v;
            if (B.f) cmacc(vf, ccast<double>(v), B.f[blk.off + r]);
        }
    }
    if (B.f) {
        vf.re = block_sum(vf.re, shd);
        vf.im = block_sum(vf.im, shd);
        if (threadIdx.x == 0) B.pvf[(long long)b * MAXCH + c] = vf;
    } else {
        __syncthreads();
    }
}

// C: tile t of the trailing region [i+1, n)^2 (lower triangle, absolute 64-tiles):
//   A -= v_{i-1} w_{i-1}^H + w_{i-1} v_{i-1}^H  (pending, i >= 1);  y partials of A v_i.
template <typename R>
__device__ void trd_phase_c(const TrdBufs<R>& B, int b, int i, long long t, const cx<R>* vprev,
                            const cx<R>* vcur, TrdSmem<R>& sm) {
    const EBlk blk = B.tab[b];
    const int n = blk.n;
    const int R0 = i + 1;
    const int T = blk.T;
    const int J0 = R0 / TB;
    int ii, jj;
    tri_index(t, &ii, &jj);
    const int I = J0 + ii, J = J0 + jj;
    const bool pend = i >= 1;
    const int tid = threadIdx.x;
    const cx<R> zero = mk<R>(R(0), R(0));
    cx<R>* A = B.A + blk.soff;
    const int tx = tid & 15, ty = tid >> 4;
    // the thread's 16 tile elements are loaded first: they depend on nothing staged below
    cx<R> xv[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int rg = I * TB + ty + 16 * a;
#pragma unroll
        for (int bq = 0; bq < 4; ++bq) {
            const int cg = J * TB + tx + 16 * bq;
            xv[a][bq] = (rg < n && cg < n && cg >= R0 && rg >= cg) ? A[(long long)rg * n + cg] : zero;
        }
    }
    if (tid < 2 * TB) {
        const int which = tid / TB, q = tid % TB;
        const int g = (which == 0 ? I : J) * TB + q;
        cx<R> vv = zero, vp = zero, wp = zero;
        if (g < n && g >= R0) {
            vv = vcur[blk.off + g];
            if (pend) {
                vp = vprev[blk.off + g];
                wp = B.w[blk.off + g];
            }
        }
        sm.sv[which][q] = vv;
        sm.svp[which][q] = vp;
        sm.swp[which][q] = wp;
    }
    __syncthreads();
    cx<R> p1[4], p2[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) p1[a] = p2[a] = zero;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = ty + 16 * a;
        const int rg = I * TB + r;
#pragma unroll
        for (int bq = 0; bq < 4; ++bq) {
            const int c = tx + 16 * bq;
            const int cg = J * TB + c;
            if (rg < n && cg < n && cg >= R0 && rg >= cg) {
                cx<R> x = xv[a][bq];
                if (pend) {
                    x = x - sm.svp[0][r] * cconj(sm.swp[1][c]) - sm.swp[0][r] * cconj(sm.svp[1][c]);
                    if (rg == cg) x.im = R(0);
                    A[(long long)rg * n + cg] = x;
                }
                cmac(p1[a], x, sm.sv[1][c]);
                if (rg > cg) cmacc(p2[bq], x, sm.sv[0][r]);
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            p1[a].re += __shfl_xor_sync(0xffffffffu, p1[a].re, o);
            p1[a].im += __shfl_xor_sync(0xffffffffu, p1[a].im, o);
        }
        if (tx == 0) sm.p1s[ty + 16 * a] = p1[a];
    }
#pragma unroll
    for (int bq = 0; bq < 4; ++bq) sm.p2buf[ty][tx + 16 * bq] = p2[bq];
    __syncthreads();
    cx<R>* Y = B.ypart + blk.yoff;
    if (tid < TB) {
        cx<R> s2 = zero;
#pragma unroll
        for (int k = 0; k < 16; ++k) s2 = s2 + sm.p2buf[k][tid];
        if (I == J) {
            Y[((long long)I * T + I) * TB + tid] = sm.p1s[tid] + s2;
        } else {
            Y[((long long)I * T + J) * TB + tid] = sm.p1s[tid];
            Y[((long long)J * T + I) * TB + tid] = s2;
        }
    }
    __syncthreads();
}

// X: on rows [j+1, n) in units of DCH rows (the tile partials of a row split over the 8
// warps): y = A v_j, x_j = tau_j y; column j+1 updated by reflector j except for the alpha
// part, into bcol; f <- H_j^H f; the partials of x_j^H v_j.
template <typename R>
__device__ void trd_phase_x(const TrdBufs<R>& B, int b, int j, int c, const cx<R>* vcur, c128 (*red)[DCH],
                            double* shd, c128* shc) {
    const EBlk blk = B.tab[b];
    const int n = blk.n;
    const int t = threadIdx.x, lane = t & 31, g = t >> 5;
    const long long r = (long long)j + 1 + (long long)c * DCH + lane;
    const int T = blk.T, J0 = (j + 1) / TB;
    const cx<R>* Yb = B.ypart + blk.yoff;
    c128 y = mk<double>(0.0, 0.0);
    if (r < n) {
        const int I = (int)(r / TB), rr = (int)(r % TB);
        const cx<R>* Y = Yb + (long long)I * T * TB + rr;
#pragma unroll 4
        for (int s = J0 + g; s < T; s += PT / 32) y = y + ccast<double>(Y[(long long)s * TB]);
    }
    red[g][lane] = y;
    // y at row j+1 (needed by every row: x_{j+1} enters column j+1's update)
    c128 y1 = mk<double>(0.0, 0.0);
    {
        const int I1 = (j + 1) / TB, rr1 = (j + 1) % TB;
        for (int s = J0 + t; s < T; s += PT) y1 = y1 + ccast<double>(Yb[((long long)I1 * T + s) * TB + rr1]);
    }
    y1.re = block_sum(y1.re, shd);
    y1.im = block_sum(y1.im, shd);
    if (B.f && t < 32) {
        const int K = (n - j + CH - 1) / CH;  // phase-R chunks of rows [j, n)
        c128 pv = mk<double>(0.0, 0.0);
        for (int k = t; k < K; k += 32) pv = pv + B.pvf[(long long)b * MAXCH + k];
        pv = warp_sum(pv);
        if (t == 0) shc[3] = cconj(B.tau[blk.off + j]) * pv;
    }
    __syncthreads();
    if (t < 32) {
        const c128 tau = B.tau[blk.off + j];
        c128 p1 = mk<double>(0.0, 0.0);
        if (r < n) {
            c128 ys = red[0][lane];
#pragma unroll
            for (int k = 1; k < PT / 32; ++k) ys = ys + red[k][lane];
            const c128 x = tau * ys;
            const c128 x1 = tau * y1;
            B.x[blk.off + r] = ccast<R>(x);
            const c128 v = ccast<double>(vcur[blk.off + r]);
            cmacc(p1, x, v);
            const cx<R>* A = B.A + blk.soff;
            B.bcol[blk.off + r] = ccast<R>(ccast<double>(A[r * n + j + 1]) - v * cconj(x1) - x);
            if (B.f) B.f[blk.off + r] = B.f[blk.off + r] - shc[3] * v;
        }
        p1 = warp_sum(p1);
        if (t == 0) B.pxv[(long long)b * MAXDCH + c] = p1;
    }
    __syncthreads();
}

template <typename R> struct TrdOcc { static constexpr int value = 2; };
template <> struct TrdOcc<float> { static constexpr int value = 3; };  // FP32: 3 CTAs per SM

template <typename R>
__global__ void __launch_bounds__(PT, TrdOcc<R>::value) trd_persist_kernel(TrdBufs<R> B, int nb, int nmax, unsigned* bar,
                                                             DevStatus* status, unsigned long long wait_ns) {
    __shared__ int sn[MAXB];
    __shared__ long long pref[MAXB + 1];
    __shared__ long long wsum[PT / 32];
    __shared__ double shd[32];
    __shared__ c128 shc[4];
    __shared__ int ok_s;
    __shared__ TrdSmem<R> sm;
    __shared__ c128 red[PT / 32][DCH];
    for (int b = threadIdx.x; b < nb; b += PT) sn[b] = B.tab[b].n;
    __syncthreads();
    long long tot = unit_prefix(nb, [&](int b) -> long long { return (sn[b] + CH - 1) / CH; }, pref, wsum);
    for (long long u = blockIdx.x; u < tot; u += gridDim.x) {
        const int b = unit_block(pref, nb, u);
        trd_prologue<R>(B, b, (int)(u - pref[b]));
    }
    if (!grid_sync(bar, status, W_TRD, &ok_s, wait_ns)) return;
    for (int j = 0; j < nmax; ++j) {
        cx<R>* vcur = (j & 1) ? B.v1 : B.v0;
        const cx<R>* vprev = (j & 1) ? B.v0 : B.v1;
        tot = unit_prefix(
            nb, [&](int b) -> long long { return sn[b] - 1 >= j ? (sn[b] - j + CH - 1) / CH : 0; }, pref, wsum);
        for (long long u = blockIdx.x; u < tot; u += gridDim.x) {
            const int b = unit_block(pref, nb, u);
            trd_phase_r<R>(B, b, j, (int)(u - pref[b]), vprev, vcur, shd, shc, status);
        }
        if (!grid_sync(bar, status, W_TRD, &ok_s, wait_ns)) return;
        tot = unit_prefix(
            nb,
            [&](int b) -> long long {
                if (sn[b] - 2 < j) return 0;
                const long long T = (sn[b] + TB - 1) / TB, J0 = (j + 1) / TB;
                return (T - J0) * (T - J0 + 1) / 2;
            },
            pref, wsum);
        for (long long u = blockIdx.x; u < tot; u += gridDim.x) {
            const int b = unit_block(pref, nb, u);
            trd_phase_c<R>(B, b, j, u - pref[b], vprev, vcur, sm);
        }
        if (!grid_sync(bar, status, W_TRD, &ok_s, wait_ns)) return;
        tot = unit_prefix(
            nb, [&](int b) -> long long { return sn[b] - 2 >= j ? (sn[b] - j - 1 + DCH - 1) / DCH : 0; }, pref, wsum);
        for (long long u = blockIdx.x; u < tot; u += gridDim.x) {
            const int b = unit_block(pref, nb, u);
            trd_phase_x<R>(B, b, j, (int)(u - pref[b]), vcur, red, shd, shc);
        }
        if (!grid_sync(bar, status, W_TRD, &ok_s, wait_ns)) return;
    }
}

// ------------------------------------------------------------------ refinement phases
struct RefSmem {
    c64 uu[QNB];             // panel dot products V_p^H y of the block
    c64 su[QNB];             // T_p u or T_p^H u
    c64 ys[CH];              // chunk of the vector being transformed
    c64 pp[PT / 32][QNB];    // per-part partial dot products
    c128 red[PT / 32][DCH];  // per-warp partial matvec sums
    c128 xs[2][TB];          // FP64 matvec
    c128 p2buf[16][TB + 1];
    c128 p1s[TB];
};

__device__ __forceinline__ int n_panels(int n) { return (n - 1 + QNB - 1) / QNB; }

// On rows [r0, r0 + CH) of the block in slot b: vec -= V_p T_p^{(H)} (V_p^H vec), with
// V_p^H vec summed from the chunk dot products of parity `par` (p < 0: no update); then
// the chunk's dot products V_q^H vec for panel q into parity par ^ 1 (q < 0: none).
// V_p = reflectors p*QNB .. p*QNB + QNB - 1, reflector k stored in row k's upper part
// (v_k[k+1] = 1 stored explicitly); T_p upper triangular, row-major.
__device__ void panel_apply(const MixBufs& M, const EBlk& blk, int b, long long cbase, long long totch, int c,
                            int p, bool herm, int q, c64* vec, int par, RefSmem& sm) {
    const int n = blk.n;
    const c64* Sf = M.Sf + blk.soff;
    const int t = threadIdx.x;
    const int r = c * CH + t;
    const int nch = (n + CH - 1) / CH;
    c64 val = mk<float>(0.f, 0.f);
    if (r < n) val = vec[blk.off + r];
    if (p >= 0) {
        {  // chunk dot products of the block, split over the 8 warps
            const int j = t & 31, g = t >> 5;
            c64 s = mk<float>(0.f, 0.f);
            for (int k = g; k < nch; k += PT / 32) s = s + M.pdot[((long long)par * totch + cbase + k) * QNB + j];
            sm.pp[g][j] = s;
        }
        __syncthreads();
        if (t < QNB) {
            c64 s = sm.pp[0][t];
#pragma unroll
            for (int k = 1; k < PT / 32; ++k) s = s + sm.pp[k][t];
            sm.uu[t] = s;
        }
        __syncthreads();
        const int i0 = p * QNB;
        const int nbp = (n - 1 - i0) < QNB ? (n - 1 - i0) : QNB;
        if (t < QNB) {
            const c64* T = M.Tf + M.toff[b] + (long long)p * QNB * QNB;  // zero beyond nbp
            c64 s = mk<float>(0.f, 0.f);
            if (herm) {
#pragma unroll 8
                for (int k = 0; k < QNB; ++k)
                    if (k <= t) cmacc(s, T[k * QNB + t], sm.uu[k]);  // (T^H u)_t
            } else {
#pragma unroll 8
                for (int k = 0; k < QNB; ++k)
                    if (k >= t) cmac(s, T[t * QNB + k], sm.uu[k]);   // (T u)_t
            }
            sm.su[t] = s;
        }
        __syncthreads();
        if (r < n && r >= i0 + 1) {
            c64 acc = mk<float>(0.f, 0.f);
            const int jmax = (r - i0 - 1) < (nbp - 1) ? (r - i0 - 1) : (nbp - 1);  // r >= i0 + j + 1
#pragma unroll 8
            for (int j = 0; j < QNB; ++j)
                if (j <= jmax) cmac(acc, Sf[(long long)(i0 + j) * n + r], sm.su[j]);
            val = val - acc;
            vec[blk.off + r] = val;
        }
    }
    if (q >= 0) {
        sm.ys[t] = val;
        __syncthreads();
        const int q0 = q * QNB;
        const int nbq = (n - 1 - q0) < QNB ? (n - 1 - q0) : QNB;
        const int j = t & 31, part = t >> 5;
        c64 acc = mk<float>(0.f, 0.f);
        if (j < nbq) {
            const c64* v = Sf + (long long)(q0 + j) * n;
            const int rlo = c * CH + part * 32;
#pragma unroll 8
            for (int k = 0; k < 32; ++k) {
                const int rr = rlo + k;
                if (rr < n && rr >= q0 + j + 1) cmacc(acc, v[rr], sm.ys[part * 32 + k]);
            }
        }
        sm.pp[part][j] = acc;
        __syncthreads();
        if (t < QNB) {
            c64 s = mk<float>(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < PT / 32; ++k) s = s + sm.pp[k][t];
            M.pdot[((long long)(par ^ 1) * totch + cbase + c) * QNB + t] = s;
        }
    }
    __syncthreads();
}

// FP64 Hermitian matvec partials of S x over tile t of the lower triangle (64-tiles).
__device__ void ref_hemv_tile(const MixBufs& M, const EBlk& blk, long long t, RefSmem& sm) {
    const int n = blk.n;
    const int T = blk.T;
    int I, J;
    tri_index(t, &I, &J);
    const int tid = threadIdx.x;
    if (tid < 2 * TB) {
        const int which = tid / TB, q = tid % TB;
        const int g = (which == 0 ? I : J) * TB + q;
        sm.xs[which][q] = g < n ? M.x[blk.off + g] : mk<double>(0.0, 0.0);
    }
    __syncthreads();
    const c128* S = M.S + blk.soff;
    const int tx = tid & 15, ty = tid >> 4;
    c128 p1[4], p2[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) p1[a] = p2[a] = mk<double>(0.0, 0.0);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = ty + 16 * a;
        const int rg = I * TB + r;
#pragma unroll
        for (int bq = 0; bq < 4; ++bq) {
            const int c = tx + 16 * bq;
            const int cg = J * TB + c;
            if (rg < n && cg < n && rg >= cg) {
                c128 v = S[(long long)rg * n + cg];
                if (rg == cg) v.im = 0.0;
                cmac(p1[a], v, sm.xs[1][c]);
                if (rg > cg) cmacc(p2[bq], v, sm.xs[0][r]);
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            p1[a].re += __shfl_xor_sync(0xffffffffu, p1[a].re, o);
            p1[a].im += __shfl_xor_sync(0xffffffffu, p1[a].im, o);
        }
        if (tx == 0) sm.p1s[ty + 16 * a] = p1[a];
    }
#pragma unroll
    for (int bq = 0; bq < 4; ++bq) sm.p2buf[ty][tx + 16 * bq] = p2[bq];
    __syncthreads();
    c128* Y = M.hpart + blk.yoff;
    if (tid < TB) {
        c128 s2 = mk<double>(0.0, 0.0);
#pragma unroll
        for (int k = 0; k < 16; ++k) s2 = s2 + sm.p2buf[k][tid];
        if (I == J) {
            Y[((long long)I * T + I) * TB + tid] = sm.p1s[tid] + s2;
        } else {
            Y[((long long)I * T + J) * TB + tid] = sm.p1s[tid];
            Y[((long long)J * T + I) * TB + tid] = s2;
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(PT, 2) refine_persist_kernel(SolveBufs B, MixBufs M, int nb, int pmaxall,
                                                                const c128* F, double shift, unsigned* bar,
                                                                DevStatus* status, int maxit,
                                                                unsigned long long wait_ns) {
    __shared__ int sn[MAXB];
    __shared__ long long cbase[MAXB + 1];  // prefix of row chunks over slots (pdot rows)
    __shared__ int sdone[MAXB];
    __shared__ double sprev[MAXB];  // ||r||^2 of the previous sweep (the same in every CTA)
    __shared__ long long pref[MAXB + 1];
    __shared__ long long wsum[PT / 32];
    __shared__ double shd[32];
    __shared__ int ok_s;
    __shared__ RefSmem sm;
    const int tid = threadIdx.x;
    for (int b = tid; b < nb; b += PT) sn[b] = B.tab[b].n;
    __syncthreads();
    if (tid == 0) {
        long long acc = 0;
        for (int b = 0; b < nb; ++b) {
            cbase[b] = acc;
            acc += (sn[b] + CH - 1) / CH;
        }
        cbase[nb] = acc;
    }
    __syncthreads();
    const long long totch = cbase[nb];
    auto chunks = [&](int b) -> long long { return (sn[b] + CH - 1) / CH; };

    // x = 0, r = F, ||F||^2 (one CTA per block)
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const EBlk blk = B.tab[b];
        double s = 0.0;
        for (int k = tid; k < blk.n; k += PT) {
            const c128 f = F[blk.off + k];
            M.x[blk.off + k] = mk<double>(0.0, 0.0);
            M.r[blk.off + k] = f;
            M.r32[blk.off + k] = ccast<float>(f);
            s += cabs2(f);
        }
        s = block_sum(s, shd);
        if (tid == 0) M.fn[b] = s;
    }
    if (!grid_sync(bar, status, W_SOLVE, &ok_s, wait_ns)) return;
    for (int b = tid; b < nb; b += PT) {
        sdone[b] = (M.fn[b] == 0.0) ? 1 : 0;
        sprev[b] = 0.0;
    }
    __syncthreads();

    for (int it = 0; it < maxit; ++it) {
        int open = 0;
        for (int b = tid; b < nb; b += PT) open |= !sdone[b];
        if (!__syncthreads_or(open)) break;

        // ---- y = Q^H r: copy, then panels 0 .. pmax-1 with T^H
        long long tot = unit_prefix(nb, [&](int b) -> long long { return sdone[b] ? 0 : chunks(b); }, pref, wsum);
        for (long long u = blockIdx.x; u < tot; u += gridDim.x) {
            const int b = unit_block(pref, nb, u);
            const int c = (int)(u - pref[b]);
            const EBlk blk = B.tab[b];
            const int r = c * CH + tid;
            if (r < blk.n) M.y32[blk.off + r] = M.r32[blk.off + r];
            __syncthreads();
            panel_apply(M, blk, b, cbase[b], totch, c, -1, true, n_panels(blk.n) > 0 ? 0 : -1, M.y32, 1, sm);
        }
        if (!grid_sync(bar, status, W_SOLVE, &ok_s, wait_ns)) return;
        for (int s = 0; s < pmaxall; ++s) {
            tot = unit_prefix(
                nb, [&](int b) -> long long { return (!sdone[b] && s < n_panels(sn[b])) ? chunks(b) : 0; }, pref,
                wsum);
            for (long long u = blockIdx.x; u < tot; u += gridDim.x) {
                const int b = unit_block(pref, nb, u);
                const EBlk blk = B.tab[b];
                const int q = s + 1 < n_panels(blk.n) ? s + 1 : -1;
                panel_apply(M, blk, b, cbase[b], totch, (int)(u - pref[b]), s, true, q, M.y32, s & 1, sm);
            }
            if (!grid_sync(bar, status, W_SOLVE, &ok_s, wait_ns)) return;
        }

        // ---- w = (T + lambda I)^{-1} y by the LDL^T factors (one thread per block)
        for (int b = blockIdx.x; b < nb; b += gridDim.x) {
            if (sdone[b] || tid != 0) continue;
            const EBlk blk = B.tab[b];
            const int n = blk.n;
            const double* piv = M.piv + blk.off;
            const double* l = M.lmul + blk.off;
            const c64* y = M.y32 + blk.off;
            c64* w = M.w32 + blk.off;
            c128 uacc = mk<double>(0.0, 0.0);
            for (int k = 0; k < n; ++k) {
                const c128 yk = ccast<double>(y[k]);
                uacc = (k == 0) ? yk : yk - l[k - 1] * uacc;
                w[k] = ccast<float>(uacc);
            }
            c128 z = (1.0 / piv[n - 1]) * ccast<double>(w[n - 1]);
            w[n - 1] = ccast<float>(z);
            for (int k = n - 2; k >= 0; --k) {
                z = (1.0 / piv[k]) * ccast<double>(w[k]) - l[k] * z;
                w[k] = ccast<float>(z);
            }
        }
        if (!grid_sync(bar, status, W_SOLVE, &ok_s, wait_ns)) return;

        // ---- x += Q w: panels pmax-1 .. 0 with T
        tot = unit_prefix(nb, [&](int b) -> long long { return sdone[b] ? 0 : chunks(b); }, pref, wsum);
        for (long long u = blockIdx.x; u < tot; u += gridDim.x) {
            const int b = unit_block(pref, nb, u);
            const int c = (int)(u - pref[b]);
            const EBlk blk = B.tab[b];
            const int np_b = n_panels(blk.n);
            panel_apply(M, blk, b, cbase[b], totch, c, -1, false, np_b - 1, M.w32, 1, sm);
            const int r = c * CH + tid;
            if (np_b == 0 && r < blk.n) M.x[blk.off + r] = M.x[blk.off + r] + ccast<double>(M.w32[blk.off + r]);
        }
        if (!grid_sync(bar, status, W_SOLVE, &ok_s, wait_ns)) return;
        for (int s = 0; s < pmaxall; ++s) {
            tot = unit_prefix(
                nb, [&](int b) -> long long { return (!sdone[b] && s < n_panels(sn[b])) ? chunks(b) : 0; }, pref,
                wsum);
            for (long long u = blockIdx.x; u < tot; u += gridDim.x) {
                const int b = unit_block(pref, nb, u);
                const int c = (int)(u - pref[b]);
                const EBlk blk = B.tab[b];
                const int p = n_panels(blk.n) - 1 - s;
                panel_apply(M, blk, b, cbase[b], totch, c, p, false, p - 1, M.w32, s & 1, sm);
                const int r = c * CH + tid;
                if (p == 0 && r < blk.n) M.x[blk.off + r] = M.x[blk.off + r] + ccast<double>(M.w32[blk.off + r]);
            }
            if (!grid_sync(bar, status, W_SOLVE, &ok_s, wait_ns)) return;
        }

        // ---- FP64 residual r = F - (S + lambda I) x
        tot = unit_prefix(
            nb,
            [&](int b) -> long long {
                const long long T = (sn[b] + TB - 1) / TB;
                return sdone[b] ? 0 : T * (T + 1) / 2;
            },
            pref, wsum);
        for (long long u = blockIdx.x; u < tot; u += gridDim.x) {
            const int b = unit_block(pref, nb, u);
            ref_hemv_tile(M, B.tab[b], u - pref[b], sm);
        }
        if (!grid_sync(bar, status, W_SOLVE, &ok_s, wait_ns)) return;
        tot = unit_prefix(
            nb, [&](int b) -> long long { return sdone[b] ? 0 : (sn[b] + DCH - 1) / DCH; }, pref, wsum);
        for (long long u = blockIdx.x; u < tot; u += gridDim.x) {
            const int b = unit_block(pref, nb, u);
            const int c = (int)(u - pref[b]);
            const EBlk blk = B.tab[b];
            const int n = blk.n;
            const int lane = tid & 31, g = tid >> 5;
            const int r = c * DCH + lane;
            c128 y = mk<double>(0.0, 0.0);
            if (r < n) {
                const int T = blk.T, I = r / TB, rr = r % TB;
                const c128* Y = M.hpart + blk.yoff + (long long)I * T * TB + rr;
#pragma unroll 4
                for (int k = g; k < T; k += PT / 32) y = y + Y[(long long)k * TB];
            }
            sm.red[g][lane] = y;
            __syncthreads();
            if (tid < 32) {
                double s = 0.0;
                if (r < n) {
                    c128 ys = sm.red[0][lane];
#pragma unroll
                    for (int k = 1; k < PT / 32; ++k) ys = ys + sm.red[k][lane];
                    const c128 x = M.x[blk.off + r];
                    const c128 res = F[blk.off + r] - ys - shift * x;
                    M.r[blk.off + r] = res;
                    M.r32[blk.off + r] = ccast<float>(res);
                    s = cabs2(res);
                }
                s = warp_sum(s);
                if (tid == 0) M.rn[(long long)b * MAXDCH + c] = s;
            }
            __syncthreads();
        }
        if (!grid_sync(bar, status, W_SOLVE, &ok_s, wait_ns)) return;

        // ---- convergence (every CTA decides the same from the same partials)
        for (int b = tid >> 5; b < nb; b += PT / 32) {  // one warp per block
            if (sdone[b]) continue;
            const int nch = (sn[b] + DCH - 1) / DCH;
            double s = 0.0;
            for (int c = tid & 31; c < nch; c += 32) s += M.rn[(long long)b * MAXDCH + c];
            s = warp_sum(s);
            if ((tid & 31) == 0) {
                // a block that does not converge (or turns non-finite) keeps done = 0: the host
                // then solves every block by the FP64 path (under capture: NQS_ERR_RETRY).
                // Below REF_FLOOR ||F|| a residual that has stopped contracting is at the FP64
                // residual's rounding floor and is accepted.
                if (s <= REF_TOL * REF_TOL * M.fn[b] ||
                    (it >= 1 && s <= REF_FLOOR * REF_FLOOR * M.fn[b] && s > 0.0625 * sprev[b]))
                    sdone[b] = 1;
                sprev[b] = s;
            }
        }
        __syncthreads();
    }
    if (blockIdx.x == 0)
        for (int b = tid; b < nb; b += PT) M.done[b] = sdone[b];
}

int coop_grid(const void* fn, int smem, int cap_per_sm, int* grid) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NQS_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NQS_ERR_CUDA;
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
        return NQS_ERR_UNSUPPORTED;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, PT, smem) != cudaSuccess || per < 1)
        return NQS_ERR_CUDA;
    *grid = sms * (per < cap_per_sm ? per : cap_per_sm);
    return NQS_OK;
}

}  // namespace

template <typename R>
int launch_trd_persist(const TrdBufs<R>& B, const EBTab& tab, unsigned* bar, DevStatus* status, cudaStream_t st) {
    int nmax = 0;
    for (int j = 0; j < tab.nb; ++j) nmax = tab.b[j].n > nmax ? tab.b[j].n : nmax;
    int grid = 0;
    const void* fn = (const void*)trd_persist_kernel<R>;
    int rc = coop_grid(fn, 0, TrdOcc<R>::value, &grid);
    if (rc) return rc;
    if (cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st) != cudaSuccess) return NQS_ERR_CUDA;
    TrdBufs<R> Bc = B;
    int nb = tab.nb;
    unsigned long long wait_ns = limits().wait_ns;
    void* args[] = {&Bc, &nb, &nmax, &bar, &status, &wait_ns};
    count_launch();
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(PT), args, 0, st) == cudaSuccess ? NQS_OK : NQS_ERR_CUDA;
}
template int launch_trd_persist<float>(const TrdBufs<float>&, const EBTab&, unsigned*, DevStatus*, cudaStream_t);
template int launch_trd_persist<double>(const TrdBufs<double>&, const EBTab&, unsigned*, DevStatus*, cudaStream_t);

int launch_refine_persist(const SolveBufs& B, const MixBufs& M, const EBTab& tab, const c128* F, double shift,
                          unsigned* bar, DevStatus* status, cudaStream_t st) {
    int pmax = 0;
    for (int j = 0; j < tab.nb; ++j) {
        const int p = (tab.b[j].n - 1 + QNB - 1) / QNB;
        pmax = p > pmax ? p : pmax;
    }
    int grid = 0;
    const void* fn = (const void*)refine_persist_kernel;
    int rc = coop_grid(fn, 0, 2, &grid);
    if (rc) return rc;
    if (cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st) != cudaSuccess) return NQS_ERR_CUDA;
    SolveBufs Bc = B;
    MixBufs Mc = M;
    int nb = tab.nb;
    const Limits lim = limits();
    int maxit = lim.ref_maxit;
    unsigned long long wait_ns = lim.wait_ns;
    void* args[] = {&Bc, &Mc, &nb, &pmax, (void*)&F, &shift, &bar, &status, &maxit, &wait_ns};
    count_launch();
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(PT), args, 0, st) == cudaSuccess ? NQS_OK : NQS_ERR_CUDA;
}

}  // namespace nqs
