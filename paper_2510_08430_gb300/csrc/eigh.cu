// Per-block shifted pseudo-inverse solve in FP64 (Sec. 2, block-layer paragraph,
// and the pseudo-inverse remark after Eq. 2):
//   S~_b = S_b + lambda I = U diag(sigma) U^H,  dtheta_b = -eta U diag(keep/sigma) U^H F_b.
//
// The eigen-decomposition is computed in factored form U = Q Z:
//  1. Householder reduction Q^H S_b Q = T (real symmetric tridiagonal), batched over
//     all blocks, one column per step. Each step fuses the rank-2 update of the
//     previous column with the Hermitian matrix-vector product of the current one,
//     so the trailing lower triangle is read and written once per column; Q^H F_b is
//     accumulated on the fly. Reflector k is stored in the (unused) upper part of
//     row k of S_b.
//  2. Eigenvalues of T + lambda I by Sturm-count bisection (sigma_max, and all of
//     them when requested); the cutoff keeps sigma_i > cutoff * sigma_max (relative)
//     or > cutoff (absolute).
//  3. If every eigenvalue is kept, pinv = inverse and z = (T + lambda I)^{-1} Q^H F_b
//     by an LDL^T tridiagonal solve (T + lambda I is positive definite then).
//     Otherwise the eigenvectors Z of T come from implicit QL iterations with
//     Wilkinson shifts and z = Z diag(keep/sigma) Z^T Q^H F_b.
//  4. dtheta_b = -eta Q z by applying the reflectors in reverse order.
#include "internal.cuh"

namespace nqs {

constexpr int TB = 64;       // tile of the fused update + matvec
constexpr int CH = 256;      // rows per CTA in the vector kernels
constexpr int MAXCH = 512;   // max row chunks per block (n <= 131072)
constexpr int QL_MAXN = 12000;

struct EBlk {
    long long off;    // offset of the block in length-n_p arrays
    long long soff;   // offset of S_b in the packed matrix array
    long long yoff;   // offset of the block's matvec partials
    int n;
    int T;            // ceil(n / TB)
    int orig;         // index of the block in the caller's order
    int pad;
};
struct EBTab {
    int nb;
    EBlk b[MAXB];
};
struct HouseP {       // per-block scalars of the current reflector
    c128 scale;       // 1 / (alpha - beta)
    c128 tau;
};
struct BlkInfo {
    double sigma_max;
    double thr;
    int n_dropped;
    int n_kept;
};

struct SolveLayout {
    size_t tab, d, e, e2, tau, f, v0, v1, w, x, z, ev, hp, info, pnorm, pvf, pxv, ypart, zmat, total;
};

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

static SolveLayout solve_layout(const int64_t* off, int nb) {
    SolveLayout L{};
    const long long np = off[nb];
    long long ytot = 0, ztot = 0;
    for (int b = 0; b < nb; ++b) {
        const long long n = off[b + 1] - off[b];
        const long long T = (n + TB - 1) / TB;
        ytot += T * T * TB;
        ztot += n * n;
    }
    size_t p = 0;
    auto take = [&](size_t bytes) { size_t at = p; p += al(bytes); return at; };
    L.tab = take(sizeof(EBlk) * (size_t)(nb > 0 ? nb : 1));
    L.d = take(8 * np);
    L.e = take(8 * np);
    L.e2 = take(8 * np);
    L.tau = take(16 * np);
    L.f = take(16 * np);
    L.v0 = take(16 * np);
    L.v1 = take(16 * np);
    L.w = take(16 * np);
    L.x = take(16 * np);
    L.z = take(16 * np);
    L.ev = take(8 * np);
    L.hp = take(sizeof(HouseP) * nb);
    L.info = take(sizeof(BlkInfo) * nb);
    L.pnorm = take(8ull * nb * MAXCH);
    L.pvf = take(16ull * nb * MAXCH);
    L.pxv = take(16ull * nb * MAXCH);
    L.ypart = take(16ull * ytot);
    L.zmat = take(8ull * ztot);
    L.total = p;
    return L;
}


struct SolveBufs {
    const EBlk* tab;
    c128* S;
    double *d, *e, *e2, *ev;
    c128 *tau, *f, *v0, *v1, *w, *x, *z;
    HouseP* hp;
    BlkInfo* info;
    double* pnorm;
    c128 *pvf, *pxv, *ypart;
    double* zmat;
};

// Views used by the Householder reduction in precision R (FP64 exact path,
// FP32 preconditioner of the mixed path). f == nullptr skips the Q^H F update.
template <typename R> struct TrdBufs {
    const EBlk* tab;
    cx<R>* A;
    cx<R> *v0, *v1, *w, *x, *ypart;
    c128* f;
    double *d, *e, *e2, *pnorm;
    c128 *tau, *pvf, *pxv;
    HouseP* hp;
};

__global__ void upload_tab_kernel(const EBTab tab, EBlk* dst) {
    for (int i = threadIdx.x; i < tab.nb; i += blockDim.x) dst[i] = tab.b[i];
}

// Copy F_b into the working vector f (later overwritten by Q^H F_b).
__global__ void init_f_kernel(const c128* __restrict__ F, long long np, c128* __restrict__ f) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x)
        f[p] = F[p];
}

// K1: bring column i up to date (rank-2 update of step i-1), partial norms of rows >= i+2.
template <typename R>
__global__ void __launch_bounds__(CH) trd_col_kernel(TrdBufs<R> B, int i, const cx<R>* __restrict__ vprev) {
    __shared__ double sh[32];
    const EBlk blk = B.tab[blockIdx.y];
    const int n = blk.n;
    if (i > n - 1) return;
    const long long r = (long long)i + (long long)blockIdx.x * CH + threadIdx.x;
    if ((long long)i + (long long)blockIdx.x * CH >= n) return;  // whole CTA past the end
    cx<R>* A = B.A + blk.soff;
    double nrm = 0.0;
    if (r < n) {
        cx<R> a = A[r * n + i];
        if (i >= 1) {
            const cx<R>* vp = vprev + blk.off;
            const cx<R>* wp = B.w + blk.off;
            const cx<R> vpi = vp[i], wpi = wp[i];
            const cx<R> vr = vp[r], wr = wp[r];
            a = a - vr * cconj(wpi) - wr * cconj(vpi);
        }
        if (r == i) a.im = R(0);
        A[r * n + i] = a;
        if (r >= i + 2) nrm = (double)cabs2(a);
    }
    nrm = block_sum(nrm, sh);
    if (threadIdx.x == 0) B.pnorm[(long long)blockIdx.y * MAXCH + blockIdx.x] = nrm;
}

// K2: Householder reflector of column i (LAPACK-style: beta real, H^H [alpha; x] = [beta; 0]).
template <typename R>
__global__ void trd_house_kernel(TrdBufs<R> B, int i, DevStatus* status) {
    const EBlk blk = B.tab[blockIdx.x];
    const int n = blk.n;
    if (i > n - 1) return;
    const cx<R>* A = B.A + blk.soff;
    const int lane = threadIdx.x;
    const int my_nch = (n - i + CH - 1) / CH;  // chunks written by trd_col_kernel for this block
    double xn = 0.0;
    for (int c = lane; c < my_nch; c += 32) xn += B.pnorm[(long long)blockIdx.x * MAXCH + c];
    xn = warp_sum(xn);
    if (lane != 0) return;
    B.d[blk.off + i] = (double)A[(long long)i * n + i].re;
    if (i > n - 2) return;
    const c128 alpha = ccast<double>(A[(long long)(i + 1) * n + i]);
    HouseP h;
    double beta;
    if (xn == 0.0 && alpha.im == 0.0) {
        beta = alpha.re;
        h.tau = mk<double>(0.0, 0.0);
        h.scale = mk<double>(0.0, 0.0);
    } else {
        const double nrm = sqrt(alpha.re * alpha.re + alpha.im * alpha.im + xn);
        beta = (alpha.re >= 0.0) ? -nrm : nrm;
        h.tau = mk<double>((beta - alpha.re) / beta, -alpha.im / beta);
        const c128 dnm = mk<double>(alpha.re - beta, alpha.im);
        const double q = cabs2(dnm);
        h.scale = mk<double>(dnm.re / q, -dnm.im / q);
    }
    if (!isfinite(beta) || !finite_cx(h.tau) || !finite_cx(h.scale))
        set_status(status, NQS_ERR_NONFINITE, W_TRD, (long long)blk.orig * 1000000 + i);
    B.e[blk.off + i] = beta;
    B.e2[blk.off + i] = beta * beta;
    B.tau[blk.off + i] = h.tau;
    B.hp[blockIdx.x] = h;
}

// K3: form v (v[i+1] = 1), store it in vcur and in row i's upper part; partial v^H f.
template <typename R>
__global__ void __launch_bounds__(CH) trd_v_kernel(TrdBufs<R> B, int i, cx<R>* __restrict__ vcur) {
    __shared__ double sh[32];
    const EBlk blk = B.tab[blockIdx.y];
    const int n = blk.n;
    if (i > n - 2) return;
    const long long base = (long long)i + 1 + (long long)blockIdx.x * CH;
    if (base >= n) return;
    const long long r = base + threadIdx.x;
    cx<R>* A = B.A + blk.soff;
    const HouseP h = B.hp[blockIdx.y];
    const cx<R> scale = ccast<R>(h.scale);
    c128 vf = mk<double>(0.0, 0.0);
    if (r < n) {
        const cx<R> v = (r == i + 1) ? mk<R>(R(1), R(0)) : A[r * n + i] * scale;
        vcur[blk.off + r] = v;
        A[(long long)i * n + r] = v;
        if (B.f) cmacc(vf, ccast<double>(v), B.f[blk.off + r]);
    }
    if (B.f) {
        vf.re = block_sum(vf.re, sh);
        vf.im = block_sum(vf.im, sh);
        if (threadIdx.x == 0) B.pvf[(long long)blockIdx.y * MAXCH + blockIdx.x] = vf;
    }
}

// K4: on the trailing region [i+1, n)^2 (lower triangle, absolute 64-tiles):
//   A -= v_{i-1} w_{i-1}^H + w_{i-1} v_{i-1}^H      (pending update, if i >= 1)
//   y  = A v_i                                        (Hermitian matvec partials)
template <typename R>
__global__ void __launch_bounds__(256) trd_fused_kernel(TrdBufs<R> B, int i, const cx<R>* __restrict__ vprev,
                                                         const cx<R>* __restrict__ vcur) {
    __shared__ cx<R> sv[2][TB], svp[2][TB], swp[2][TB];
    __shared__ cx<R> p2buf[16][TB + 1];
    __shared__ cx<R> p1s[TB];
    const EBlk blk = B.tab[blockIdx.y];
    const int n = blk.n;
    if (i > n - 2) return;
    const int R0 = i + 1;
    const int T = blk.T;
    const int J0 = R0 / TB;
    const long long cnt = (long long)(T - J0) * (T - J0 + 1) / 2;
    const long long t = blockIdx.x;
    if (t >= cnt) return;
    long long ii = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
    while (ii * (ii + 1) / 2 > t) --ii;
    const int I = J0 + (int)ii;
    const int J = J0 + (int)(t - ii * (ii + 1) / 2);
    const bool pend = i >= 1;
    const int tid = threadIdx.x;
    const cx<R> zero = mk<R>(R(0), R(0));
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
        sv[which][q] = vv;
        svp[which][q] = vp;
        swp[which][q] = wp;
    }
    __syncthreads();
    cx<R>* A = B.A + blk.soff;
    const int tx = tid & 15, ty = tid >> 4;
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
                const long long idx = (long long)rg * n + cg;
                cx<R> x = A[idx];
                if (pend) {
                    x = x - svp[0][r] * cconj(swp[1][c]) - swp[0][r] * cconj(svp[1][c]);
                    if (rg == cg) x.im = R(0);
                    A[idx] = x;
                }
                cmac(p1[a], x, sv[1][c]);
                if (rg > cg) cmacc(p2[bq], x, sv[0][r]);
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
        if (tx == 0) p1s[ty + 16 * a] = p1[a];
    }
#pragma unroll
    for (int bq = 0; bq < 4; ++bq) p2buf[ty][tx + 16 * bq] = p2[bq];
    __syncthreads();
    cx<R>* Y = B.ypart + blk.yoff;
    if (tid < TB) {
        cx<R> s2 = zero;
#pragma unroll
        for (int k = 0; k < 16; ++k) s2 = s2 + p2buf[k][tid];
        if (I == J) {
            Y[((long long)I * T + I) * TB + tid] = p1s[tid] + s2;
        } else {
            Y[((long long)I * T + J) * TB + tid] = p1s[tid];
            Y[((long long)J * T + I) * TB + tid] = s2;
        }
    }
}

// K5: y = sum of matvec partials, x = tau y, partial x^H v.
template <typename R>
__global__ void __launch_bounds__(CH) trd_w1_kernel(TrdBufs<R> B, int i, const cx<R>* __restrict__ vcur) {
    __shared__ double sh[32];
    const EBlk blk = B.tab[blockIdx.y];
    const int n = blk.n;
    if (i > n - 2) return;
    const long long base = (long long)i + 1 + (long long)blockIdx.x * CH;
    if (base >= n) return;
    const long long r = base + threadIdx.x;
    const c128 tau = B.hp[blockIdx.y].tau;
    c128 xv = mk<double>(0.0, 0.0);
    if (r < n) {
        const int T = blk.T, J0 = (i + 1) / TB;
        const int I = (int)(r / TB), rr = (int)(r % TB);
        const cx<R>* Y = B.ypart + blk.yoff + (long long)I * T * TB + rr;
        c128 y = mk<double>(0.0, 0.0);
        for (int s = J0; s < T; ++s) y = y + ccast<double>(Y[(long long)s * TB]);
        const c128 x = tau * y;
        B.x[blk.off + r] = ccast<R>(x);
        cmacc(xv, x, ccast<double>(vcur[blk.off + r]));
    }
    xv.re = block_sum(xv.re, sh);
    xv.im = block_sum(xv.im, sh);
    if (threadIdx.x == 0) B.pxv[(long long)blockIdx.y * MAXCH + blockIdx.x] = xv;
}

// K6: w = x - 0.5 tau (x^H v) v; f <- H^H f = f - conj(tau) v (v^H f).
template <typename R>
__global__ void __launch_bounds__(CH) trd_w2_kernel(TrdBufs<R> B, int i, const cx<R>* __restrict__ vcur) {
    __shared__ c128 red[2];
    const EBlk blk = B.tab[blockIdx.y];
    const int n = blk.n;
    if (i > n - 2) return;
    const long long base = (long long)i + 1 + (long long)blockIdx.x * CH;
    if (base >= n) return;
    if (threadIdx.x < 32) {
        const int my_nch = (n - i - 1 + CH - 1) / CH;  // chunks of rows [i+1, n)
        c128 a = mk<double>(0.0, 0.0), b = a;
        for (int c = threadIdx.x; c < my_nch; c += 32) {
            a = a + B.pxv[(long long)blockIdx.y * MAXCH + c];
            if (B.f) b = b + B.pvf[(long long)blockIdx.y * MAXCH + c];
        }
        a = warp_sum(a);
        b = warp_sum(b);
        if (threadIdx.x == 0) {
            red[0] = a;
            red[1] = b;
        }
    }
    __syncthreads();
    const long long r = base + threadIdx.x;
    if (r >= n) return;
    const c128 tau = B.hp[blockIdx.y].tau;
    const c128 alpha = (-0.5) * (tau * red[0]);
    const c128 v = ccast<double>(vcur[blk.off + r]);
    B.w[blk.off + r] = ccast<R>(ccast<double>(B.x[blk.off + r]) + alpha * v);
    if (B.f) {
        const c128 g = cconj(tau) * red[1];
        B.f[blk.off + r] = B.f[blk.off + r] - g * v;
    }
}

// Householder reduction of every block of the table (blocks sorted by size, descending).
template <typename R>
static int trd_reduce(const TrdBufs<R>& B, const EBTab& tab, cudaStream_t st, DevStatus* status) {
    int nmax = 0;
    for (int j = 0; j < tab.nb; ++j) nmax = tab.b[j].n > nmax ? tab.b[j].n : nmax;
    for (int i = 0; i < nmax; ++i) {
        int act1 = 0, act2 = 0;  // blocks with n-1 >= i, with n-2 >= i
        while (act1 < tab.nb && tab.b[act1].n - 1 >= i) ++act1;
        while (act2 < tab.nb && tab.b[act2].n - 2 >= i) ++act2;
        cx<R>* vcur = (i & 1) ? B.v1 : B.v0;
        cx<R>* vprev = (i & 1) ? B.v0 : B.v1;
        const int nch1 = (nmax - i + CH - 1) / CH;
        count_launch();
        trd_col_kernel<R><<<dim3(nch1, act1), CH, 0, st>>>(B, i, vprev);
        count_launch();
        trd_house_kernel<R><<<act1, 32, 0, st>>>(B, i, status);
        if (act2 > 0) {
            const int nch2 = (nmax - i - 1 + CH - 1) / CH;
            count_launch();
            trd_v_kernel<R><<<dim3(nch2, act2), CH, 0, st>>>(B, i, vcur);
            const int T0 = tab.b[0].T, J0 = (i + 1) / TB;
            const long long cnt = (long long)(T0 - J0) * (T0 - J0 + 1) / 2;
            count_launch();
            trd_fused_kernel<R><<<dim3((unsigned)cnt, act2), 256, 0, st>>>(B, i, vprev, vcur);
            count_launch();
            trd_w1_kernel<R><<<dim3(nch2, act2), CH, 0, st>>>(B, i, vcur);
            count_launch();
            trd_w2_kernel<R><<<dim3(nch2, act2), CH, 0, st>>>(B, i, vcur);
        }
        if (cudaGetLastError() != cudaSuccess) return NQS_ERR_CUDA;
    }
    return NQS_OK;
}

// ------------------------------------------------------------------ eigenvalues
__device__ __forceinline__ int sturm_count(const double* __restrict__ d, const double* __restrict__ e2, int n,
                                           double shift, double x, double pivmin) {
    int cnt = 0;
    double q = d[0] + shift - x;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
    for (int k = 1; k < n; ++k) {
        q = (d[k] + shift - x) - e2[k - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        cnt += q < 0.0;
    }
    return cnt;
}

__device__ void gersh(const double* d, const double* e, int n, double shift, double* lo, double* hi) {
    double gl = 1e300, gu = -1e300;
    for (int k = 0; k < n; ++k) {
        const double r = (k > 0 ? fabs(e[k - 1]) : 0.0) + (k < n - 1 ? fabs(e[k]) : 0.0);
        gl = fmin(gl, d[k] + shift - r);
        gu = fmax(gu, d[k] + shift + r);
    }
    const double span = fmax(fabs(gl), fabs(gu));
    *lo = gl - 4.0 * 2.22e-16 * span - 1e-300;
    *hi = gu + 4.0 * 2.22e-16 * span + 1e-300;
}

// k-th smallest eigenvalue (0-based) by bisection on [lo, hi].
__device__ double bisect_k(const double* d, const double* e2, int n, double shift, int k, double lo, double hi,
                           double pivmin) {
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (hi - lo <= 2.0 * 2.22e-16 * fmax(fabs(lo), fabs(hi)) + pivmin) break;
        if (sturm_count(d, e2, n, shift, mid, pivmin) <= k) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// One thread per block: sigma_max, threshold, number dropped.
__global__ void eig_bounds_kernel(SolveBufs B, int nb, SolveArgs a, DevStatus* status) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nb) return;
    const EBlk blk = B.tab[j];
    const int n = blk.n;
    const double* d = B.d + blk.off;
    const double* e = B.e + blk.off;
    const double* e2 = B.e2 + blk.off;
    double lo, hi;
    gersh(d, e, n, a.shift, &lo, &hi);
    double emax = 0.0;
    for (int k = 0; k + 1 < n; ++k) emax = fmax(emax, e2[k]);
    const double pivmin = 1e-290 * fmax(1.0, emax);
    const double smax = bisect_k(d, e2, n, a.shift, n - 1, lo, hi, pivmin);
    const double thr = a.cutoff_mode == 0 ? a.cutoff * smax : a.cutoff;
    int drop = sturm_count(d, e2, n, a.shift, thr, pivmin);
    // eigenvalues within rounding of thr count as dropped when the Sturm count says <= thr
    BlkInfo info;
    info.sigma_max = smax;
    info.thr = thr;
    info.n_dropped = drop;
    info.n_kept = n - drop;
    B.info[j] = info;
    if (!isfinite(smax)) set_status(status, NQS_ERR_NONFINITE, W_BISECT, blk.orig);
}

// All eigenvalues (ascending) by bisection, one thread per eigenvalue.
__global__ void eig_all_kernel(SolveBufs B, int nb, double shift, double* __restrict__ evals) {
    const EBlk blk = B.tab[blockIdx.y];
    const int n = blk.n;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double* d = B.d + blk.off;
    const double* e = B.e + blk.off;
    const double* e2 = B.e2 + blk.off;
    double lo, hi;
    gersh(d, e, n, shift, &lo, &hi);
    double emax = 0.0;
    for (int q = 0; q + 1 < n; ++q) emax = fmax(emax, e2[q]);
    const double pivmin = 1e-290 * fmax(1.0, emax);
    evals[blk.off + k] = bisect_k(d, e2, n, shift, k, lo, hi, pivmin);
}

// LDL^T solve of (T + shift I) z = f for blocks whose eigenvalues are all kept.
__global__ void ldl_solve_kernel(SolveBufs B, int nb, double shift, DevStatus* status) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nb) return;
    const EBlk blk = B.tab[j];
    if (B.info[j].n_dropped != 0) return;
    const int n = blk.n;
    const double* d = B.d + blk.off;
    const double* e = B.e + blk.off;
    const c128* f = B.f + blk.off;
    c128* z = B.z + blk.off;
    // scratch: the x vector of this block holds 2n doubles: pivots then multipliers
    double* piv = reinterpret_cast<double*>(B.x + blk.off);
    double* l = piv + n;
    // forward elimination
    double p = d[0] + shift;
    piv[0] = p;
    c128 u = f[0];
    z[0] = u;
    bool ok = p > 0.0;
    for (int k = 1; k < n; ++k) {
        const double lk = e[k - 1] / p;
        l[k - 1] = lk;
        p = d[k] + shift - lk * e[k - 1];
        piv[k] = p;
        ok = ok && (p > 0.0);
        u = f[k] - lk * u;
        z[k] = u;
    }
    // diagonal + back substitution
    c128 zn = (1.0 / piv[n - 1]) * z[n - 1];
    z[n - 1] = zn;
    for (int k = n - 2; k >= 0; --k) {
        zn = (1.0 / piv[k]) * z[k] - l[k] * zn;
        z[k] = zn;
    }
    if (!ok) set_status(status, NQS_ERR_NONFINITE, W_SOLVE, blk.orig);
}

// Implicit QL with Wilkinson shifts on T + shift I, eigenvectors accumulated in
// Zt (eigenvector-major, Zt[i*n + k]); then z = Z diag(keep/sigma) Z^T f.
// Thread 0 runs the scalar recurrence of a sweep; all threads apply its plane
// rotations to their rows.
__global__ void __launch_bounds__(512) ql_solve_kernel(SolveBufs B, int nb, SolveArgs a, DevStatus* status) {
    extern __shared__ __align__(16) double qsm[];
    const EBlk blk = B.tab[blockIdx.x];
    if (B.info[blockIdx.x].n_dropped == 0) return;
    const int n = blk.n;
    double* rc = qsm;          // cosines [n]
    double* rs = qsm + n;      // sines   [n]
    __shared__ int sh_lo, sh_hi, sh_flag, sh_done;
    double* dd = B.ev + blk.off;                       // working diagonal -> eigenvalues
    double* ee = reinterpret_cast<double*>(B.x + blk.off);  // working off-diagonal
    double* Zt = B.zmat + blk.soff;                    // n*n (packed like S)
    for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) Zt[q] = (q / n == q % n) ? 1.0 : 0.0;
    if (threadIdx.x == 0) {
        for (int k = 0; k < n; ++k) dd[k] = B.d[blk.off + k] + a.shift;
        for (int k = 0; k + 1 < n; ++k) ee[k] = B.e[blk.off + k];
        ee[n - 1] = 0.0;
    }
    __syncthreads();
    const int maxit = 60;
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        while (true) {
            if (threadIdx.x == 0) {
                int m = l;
                for (; m < n - 1; ++m) {
                    const double dsum = fabs(dd[m]) + fabs(dd[m + 1]);
                    if (fabs(ee[m]) <= 2.22e-16 * dsum) break;
                }
                sh_flag = 0;
                if (m == l) {
                    sh_done = 1;
                } else if (iter++ >= maxit) {
                    sh_done = 1;
                    set_status(status, NQS_ERR_NOT_CONVERGED, W_QL, blk.orig);
                } else {
                    sh_done = 0;
                    // Wilkinson shift from the leading 2x2 of the unreduced part
                    double g = (dd[l + 1] - dd[l]) / (2.0 * ee[l]);
                    double r = hypot(g, 1.0);
                    g = dd[m] - dd[l] + ee[l] / (g + copysign(r, g));
                    double s = 1.0, c = 1.0, p = 0.0;
                    int k = m - 1;
                    int lo_rot = l;
                    for (; k >= l; --k) {
                        const double f = s * ee[k];
                        const double b = c * ee[k];
                        r = hypot(f, g);
                        ee[k + 1] = r;
                        if (r == 0.0) {
                            dd[k + 1] -= p;
                            ee[m] = 0.0;
                            lo_rot = k + 1;
                            sh_flag = 1;
                            break;
                        }
                        s = f / r;
                        c = g / r;
                        g = dd[k + 1] - p;
                        r = (dd[k] - g) * s + 2.0 * c * b;
                        p = s * r;
                        dd[k + 1] = g + p;
                        g = c * r - b;
                        rc[k] = c;
                        rs[k] = s;
                    }
                    if (!sh_flag) {
                        dd[l] -= p;
                        ee[l] = g;
                        ee[m] = 0.0;
                    }
                    sh_lo = lo_rot;
                    sh_hi = m - 1;
                }
            }
            __syncthreads();
            if (sh_done) break;
            // apply rotations k = hi down to lo to eigenvector columns k, k+1
            const int lo = sh_lo, hi = sh_hi;
            for (int row = threadIdx.x; row < n; row += blockDim.x) {
                for (int k = hi; k >= lo; --k) {
                    double* zk = Zt + (long long)k * n + row;
                    double* zk1 = zk + n;
                    const double f = *zk1;
                    const double z0 = *zk;
                    *zk1 = rs[k] * z0 + rc[k] * f;
                    *zk = rc[k] * z0 - rs[k] * f;
                }
            }
            __syncthreads();
        }
        __syncthreads();
    }
    // keep decision on the QL eigenvalues
    __shared__ double s_max;
    __shared__ int s_kept;
    if (threadIdx.x == 0) {
        double mx = -1e300;
        for (int k = 0; k < n; ++k) mx = fmax(mx, dd[k]);
        s_max = mx;
        const double thr = a.cutoff_mode == 0 ? a.cutoff * mx : a.cutoff;
        int kept = 0;
        for (int k = 0; k < n; ++k) kept += dd[k] > thr;
        s_kept = kept;
        B.info[blockIdx.x].n_kept = kept;
        B.info[blockIdx.x].sigma_max = mx;
        B.info[blockIdx.x].thr = thr;
    }
    __syncthreads();
    const double thr = B.info[blockIdx.x].thr;
    // coefficients c_i = (Z_i^T f) / sigma_i for kept i (stored in rc/rs as re/im)
    const c128* f = B.f + blk.off;
    for (int iv = threadIdx.x; iv < n; iv += blockDim.x) {
        double cr = 0.0, ci = 0.0;
        if (dd[iv] > thr) {
            const double* zi = Zt + (long long)iv * n;
            for (int k = 0; k < n; ++k) {
                cr = fma(zi[k], f[k].re, cr);
                ci = fma(zi[k], f[k].im, ci);
            }
            cr /= dd[iv];
            ci /= dd[iv];
        }
        rc[iv] = cr;
        rs[iv] = ci;
    }
    __syncthreads();
    c128* z = B.z + blk.off;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double zr = 0.0, zi2 = 0.0;
        for (int iv = 0; iv < n; ++iv) {
            const double zv = Zt[(long long)iv * n + k];
            zr = fma(zv, rc[iv], zr);
            zi2 = fma(zv, rs[iv], zi2);
        }
        z[k] = mk<double>(zr, zi2);
    }
}

// dtheta_b = -eta Q z: apply H_k = I - tau_k v_k v_k^H for k = n-2 .. 0.
__global__ void __launch_bounds__(512) back_kernel(SolveBufs B, int nb, double eta, c128* __restrict__ dtheta,
                                                    int32_t* __restrict__ n_kept, DevStatus* status) {
    __shared__ double sh[32];
    const EBlk blk = B.tab[blockIdx.x];
    const int n = blk.n;
    const c128* A = B.S + blk.soff;
    c128* z = B.z + blk.off;
    for (int k = n - 2; k >= 0; --k) {
        const c128 tau = B.tau[blk.off + k];
        if (tau.re == 0.0 && tau.im == 0.0) continue;
        const c128* v = A + (long long)k * n;  // v[r] for r >= k+1
        c128 dot = mk<double>(0.0, 0.0);
        for (int r = k + 1 + threadIdx.x; r < n; r += blockDim.x) cmacc(dot, v[r], z[r]);
        dot.re = block_sum(dot.re, sh);
        dot.im = block_sum(dot.im, sh);
        const c128 g = tau * dot;
        for (int r = k + 1 + threadIdx.x; r < n; r += blockDim.x) z[r] = z[r] - g * v[r];
        __syncthreads();
    }
    bool bad = false;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const c128 o = (-eta) * z[r];
        bad |= !finite_cx(o);
        dtheta[blk.off + r] = o;
    }
    if (bad) set_status(status, NQS_ERR_NONFINITE, W_SOLVE, blk.orig);
    if (threadIdx.x == 0 && n_kept) n_kept[blk.orig] = B.info[blockIdx.x].n_kept;
}

// ------------------------------------------------------------------ mixed precision
// The O(n^3) reduction runs in FP32 on a copy of S; Q (FP32) is formed explicitly;
// (S + lambda I) x = F is then solved by iterative refinement in which every
// residual r = F - (S + lambda I) x uses the FP64 S and the correction applies the
// FP32 factorisation, x += Q (T + lambda I)^{-1} Q^H r. The iteration converges to
// the FP64 solution when the FP32 factors approximate S to better than 1/kappa.
constexpr int QNB = 32;      // reflectors per panel in the Q formation
constexpr int QT = 64;       // tile of the Q formation kernels
constexpr int REF_MAXIT = 30;
constexpr double REF_TOL = 1e-14;

struct MixBufs {
    const EBlk* tab;
    const c128* S;        // FP64 S (lower triangles), packed
    c64* Sf;              // FP32 copy, reduced in place (reflectors in the upper rows)
    c64* Q;               // explicit FP32 Q per block, packed like S
    c64* Tf;              // T factors: per block ceil((n-1)/QNB) panels x QNB x QNB
    long long* toff;      // per slot offset into Tf
    c64* W;               // per block QNB x n scratch (T V^H Q' of the current panel)
    double *d, *e;        // FP32-reduced tridiagonal (stored in FP64)
    double *piv, *lmul;   // LDL^T of T + lambda I
    c128 *x, *r;          // refinement iterate and residual (FP64)
    c64 *r32, *y32, *w32; // FP32 work vectors
    c64* ypart;           // Q^H r partial sums [chunk][np]
    c128* hpart;          // FP64 Hermitian matvec partials (T^2 x 64 per block)
    double* rn;           // per slot ||r||^2 partials [MAXCH]
    double* fn;           // per slot ||F||^2
    int* done;            // per slot converged flag
    int* fallback;        // per slot: cutoff may drop an eigenvalue (needs the FP64 path)
};

__global__ void to_fp32_kernel(const c128* __restrict__ S, long long n, c64* __restrict__ Sf) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        Sf[i] = ccast<float>(S[i]);
}

// One thread per block: FP32-based bounds; a block needs the FP64 path when an
// eigenvalue might fall on the dropped side of the cutoff within the FP32 error.
__global__ void mix_cert_kernel(SolveBufs B, MixBufs M, int nb, SolveArgs a, DevStatus* status) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nb) return;
    const EBlk blk = B.tab[j];
    const int n = blk.n;
    const double* d = M.d + blk.off;
    const double* e = M.e + blk.off;
    const double* e2 = B.e2 + blk.off;
    double lo, hi;
    gersh(d, e, n, a.shift, &lo, &hi);
    double emax = 0.0;
    for (int k = 0; k + 1 < n; ++k) emax = fmax(emax, e2[k]);
    const double pivmin = 1e-290 * fmax(1.0, emax);
    const double smax = bisect_k(d, e2, n, a.shift, n - 1, lo, hi, pivmin);
    const double smin = bisect_k(d, e2, n, a.shift, 0, lo, hi, pivmin);
    const double err = 4e-5 * fabs(smax);  // bound on the FP32 reduction's eigenvalue error
    const double thr_hi = a.cutoff_mode == 0 ? a.cutoff * (smax + err) : a.cutoff;
    // a Gram matrix plus shift has no eigenvalue below shift beyond its own rounding
    const double lower = a.psd ? fmax(smin - err, a.shift - 1e-6 * fabs(smax)) : smin - err;
    M.fallback[j] = (lower > thr_hi && lower > 0.0) ? 0 : 1;
    BlkInfo info;
    info.sigma_max = smax;
    info.thr = a.cutoff_mode == 0 ? a.cutoff * smax : a.cutoff;
    info.n_dropped = 0;
    info.n_kept = n;
    B.info[j] = info;
    if (!isfinite(smax)) set_status(status, NQS_ERR_NONFINITE, W_BISECT, blk.orig);
    // LDL^T of T + shift I (positive definite when no eigenvalue is dropped)
    double* piv = M.piv + blk.off;
    double* l = M.lmul + blk.off;
    double p = d[0] + a.shift;
    piv[0] = p;
    for (int k = 1; k < n; ++k) {
        const double lk = e[k - 1] / p;
        l[k - 1] = lk;
        p = d[k] + a.shift - lk * e[k - 1];
        piv[k] = p;
    }
}

// T factor of each panel (forward, columnwise): T[j][j] = tau_j,
// T[0:j, j] = -tau_j T[0:j, 0:j] (V[:, 0:j]^H v_j), V = reflectors i0 .. i0+nbp-1.
__global__ void __launch_bounds__(256) qt_factor_kernel(SolveBufs B, MixBufs M) {
    __shared__ c128 G[QNB][QNB + 1];
    __shared__ c128 Ts[QNB][QNB + 1];
    const EBlk blk = B.tab[blockIdx.y];
    const int n = blk.n;
    const int p = blockIdx.x;
    const int i0 = p * QNB;
    if (i0 >= n - 1) return;
    const int nbp = (n - 1 - i0) < QNB ? (n - 1 - i0) : QNB;
    const c64* A = M.Sf + blk.soff;
    // G = V^H V over rows r in [i0+1, n); V[r][j] = A[(i0+j) n + r] for r >= i0+j+1, else 0
    for (int idx = threadIdx.x; idx < nbp * nbp; idx += blockDim.x) {
        const int a = idx / nbp, b = idx % nbp;
        if (b < a) continue;
        c128 acc = mk<double>(0.0, 0.0);
        const int r0 = i0 + b + 1;  // both vectors nonzero from max(a, b) + i0 + 1
        const c64* va = A + (long long)(i0 + a) * n;
        const c64* vb = A + (long long)(i0 + b) * n;
        for (int r = r0; r < n; ++r) cmacc(acc, ccast<double>(va[r]), ccast<double>(vb[r]));
        G[a][b] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 0; j < nbp; ++j) {
            const c128 tj = B.tau[blk.off + i0 + j];
            for (int a = 0; a < j; ++a) {
                c128 s = mk<double>(0.0, 0.0);
                for (int b = a; b < j; ++b) cmac(s, Ts[a][b], G[b][j]);
                Ts[a][j] = mk<double>(0.0, 0.0) - tj * s;
            }
            Ts[j][j] = tj;
            for (int a = j + 1; a < nbp; ++a) Ts[a][j] = mk<double>(0.0, 0.0);
        }
    }
    __syncthreads();
    c64* T = M.Tf + M.toff[blockIdx.y] + (long long)p * QNB * QNB;
    for (int idx = threadIdx.x; idx < QNB * QNB; idx += blockDim.x) {
        const int a = idx / QNB, b = idx % QNB;
        T[idx] = (a < nbp && b < nbp) ? ccast<float>(Ts[a][b]) : mk<float>(0.f, 0.f);
    }
}

__global__ void q_identity_kernel(SolveBufs B, MixBufs M) {
    const EBlk blk = B.tab[blockIdx.y];
    const long long nn = (long long)blk.n * blk.n;
    c64* Q = M.Q + blk.soff;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x)
        Q[i] = (i / blk.n == i % blk.n) ? mk<float>(1.f, 0.f) : mk<float>(0.f, 0.f);
}

// W[:, c-tile] = T (V^H Q'[:, c-tile]) for panel p; Q' = Q[i0+1:, i0+1:].
__global__ void __launch_bounds__(256) q_w_kernel(SolveBufs B, MixBufs M, int p) {
    __shared__ c64 Vs[32][QNB + 1];
    __shared__ c64 Qs[32][QT + 1];
    __shared__ c64 Ws[QNB][QT + 1];
    const EBlk blk = B.tab[blockIdx.y];
    const int n = blk.n;
    const int i0 = p * QNB;
    if (i0 >= n - 1) return;
    const int nbp = (n - 1 - i0) < QNB ? (n - 1 - i0) : QNB;
    const int m = n - i0 - 1;
    const int c0 = blockIdx.x * QT;
    if (c0 >= m) return;
    const c64* A = M.Sf + blk.soff;
    const c64* Q = M.Q + blk.soff;
    const int tid = threadIdx.x;
    // thread -> (j = tid / 8 in [0,32), columns cc = tid % 8 + 8 q, q = 0..7)
    const int jj = tid >> 3, cl = tid & 7;
    c64 acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = mk<float>(0.f, 0.f);
    for (int r0 = 0; r0 < m; r0 += 32) {
        for (int idx = tid; idx < 32 * QNB; idx += 256) {
            const int rr = idx / QNB, j = idx % QNB;
            const int r = r0 + rr;  // local row in [0, m): global row i0 + 1 + r
            c64 v = mk<float>(0.f, 0.f);
            if (r < m && j < nbp && r >= j) v = A[(long long)(i0 + j) * n + (i0 + 1 + r)];
            Vs[rr][j] = v;
        }
        for (int idx = tid; idx < 32 * QT; idx += 256) {
            const int rr = idx / QT, c = idx % QT;
            const int r = r0 + rr;
            c64 v = mk<float>(0.f, 0.f);
            if (r < m && c0 + c < m) v = Q[(long long)(i0 + 1 + r) * n + (i0 + 1 + c0 + c)];
            Qs[rr][c] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
            const c64 v = Vs[rr][jj];
#pragma unroll
            for (int q = 0; q < 8; ++q) cmacc(acc[q], v, Qs[rr][cl + 8 * q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) Ws[jj][cl + 8 * q] = acc[q];
    __syncthreads();
    // W = T Ws (T upper triangular, QNB x QNB)
    const c64* T = M.Tf + M.toff[blockIdx.y] + (long long)p * QNB * QNB;
    c64* Wout = M.W + (long long)blk.off * QNB;  // [QNB][n] per block
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int c = cl + 8 * q;
        c64 s = mk<float>(0.f, 0.f);
        for (int b = jj; b < QNB; ++b) cmac(s, T[jj * QNB + b], Ws[b][c]);
        if (c0 + c < m) Wout[(long long)jj * n + c0 + c] = s;
    }
}

// Q'[r-tile, c-tile] -= V[r-tile, :] W[:, c-tile]
__global__ void __launch_bounds__(256) q_update_kernel(SolveBufs B, MixBufs M, int p) {
    __shared__ c64 Vs[QT][QNB + 1];
    __shared__ c64 Ws[QNB][QT + 1];
    const EBlk blk = B.tab[blockIdx.z];
    const int n = blk.n;
    const int i0 = p * QNB;
    if (i0 >= n - 1) return;
    const int nbp = (n - 1 - i0) < QNB ? (n - 1 - i0) : QNB;
    const int m = n - i0 - 1;
    const int r0 = blockIdx.y * QT, c0 = blockIdx.x * QT;
    if (r0 >= m || c0 >= m) return;
    const c64* A = M.Sf + blk.soff;
    c64* Q = M.Q + blk.soff;
    const c64* Win = M.W + (long long)blk.off * QNB;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < QT * QNB; idx += 256) {
        const int rr = idx / QNB, j = idx % QNB;
        const int r = r0 + rr;
        c64 v = mk<float>(0.f, 0.f);
        if (r < m && j < nbp && r >= j) v = A[(long long)(i0 + j) * n + (i0 + 1 + r)];
        Vs[rr][j] = v;
    }
    for (int idx = tid; idx < QNB * QT; idx += 256) {
        const int j = idx / QT, c = idx % QT;
        Ws[j][c] = (c0 + c < m && j < nbp) ? Win[(long long)j * n + c0 + c] : mk<float>(0.f, 0.f);
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int rr = ty + 16 * a;
        const int r = r0 + rr;
        if (r >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int cc = tx + 16 * b;
            const int c = c0 + cc;
            if (c >= m) continue;
            c64 s = mk<float>(0.f, 0.f);
#pragma unroll 8
            for (int j = 0; j < QNB; ++j) cmac(s, Vs[rr][j], Ws[j][cc]);
            const long long idx = (long long)(i0 + 1 + r) * n + (i0 + 1 + c);
            Q[idx] = Q[idx] - s;
        }
    }
}

// Refinement init: x = 0, r = F, ||F||^2.
__global__ void ref_init_kernel(SolveBufs B, MixBufs M, const c128* __restrict__ F) {
    __shared__ double sh[32];
    const EBlk blk = B.tab[blockIdx.x];
    double s = 0.0;
    for (int k = threadIdx.x; k < blk.n; k += blockDim.x) {
        const c128 f = F[blk.off + k];
        M.x[blk.off + k] = mk<double>(0.0, 0.0);
        M.r[blk.off + k] = f;
        M.r32[blk.off + k] = ccast<float>(f);
        s += cabs2(f);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        M.fn[blockIdx.x] = s;
        M.done[blockIdx.x] = (s == 0.0) ? 1 : 0;
    }
}

// y partials over 256-row chunks: ypart[chunk][off + j] = sum_{i in chunk} conj(Q[i][j]) r32[i]
__global__ void __launch_bounds__(256) ref_qh_kernel(SolveBufs B, MixBufs M, long long np) {
    __shared__ c64 rs[256];
    const EBlk blk = B.tab[blockIdx.z];
    if (M.done[blockIdx.z] || M.fallback[blockIdx.z]) return;
    const int n = blk.n;
    const int i0 = blockIdx.y * 256;
    if (i0 >= n || (int)(blockIdx.x * 256) >= n) return;
    const int i1 = (i0 + 256) < n ? (i0 + 256) : n;
    if (i0 + (int)threadIdx.x < n) rs[threadIdx.x] = M.r32[blk.off + i0 + threadIdx.x];
    __syncthreads();
    const int j = blockIdx.x * 256 + threadIdx.x;
    if (j >= n) return;
    const c64* Q = M.Q + blk.soff;
    c64 acc = mk<float>(0.f, 0.f);
    for (int i = i0; i < i1; ++i) cmacc(acc, Q[(long long)i * n + j], rs[i - i0]);
    M.ypart[(long long)blockIdx.y * np + blk.off + j] = acc;
}

// w = (T + shift I)^{-1} (sum of the y partials), one thread per block (sequential LDL^T solve).
__global__ void ref_tri_kernel(SolveBufs B, MixBufs M, int nb, long long np) {
    const int jb = blockIdx.x * blockDim.x + threadIdx.x;
    if (jb >= nb) return;
    if (M.done[jb] || M.fallback[jb]) return;
    const EBlk blk = B.tab[jb];
    const int n = blk.n;
    const int nch = (n + 255) / 256;
    const double* piv = M.piv + blk.off;
    const double* l = M.lmul + blk.off;
    c64* w = M.w32 + blk.off;
    c128 u = mk<double>(0.0, 0.0);
    for (int k = 0; k < n; ++k) {
        c128 y = mk<double>(0.0, 0.0);
        for (int c = 0; c < nch; ++c) y = y + ccast<double>(M.ypart[(long long)c * np + blk.off + k]);
        u = (k == 0) ? y : y - l[k - 1] * u;
        w[k] = ccast<float>(u);  // forward-eliminated values
    }
    c128 z = (1.0 / piv[n - 1]) * ccast<double>(w[n - 1]);
    w[n - 1] = ccast<float>(z);
    for (int k = n - 2; k >= 0; --k) {
        z = (1.0 / piv[k]) * ccast<double>(w[k]) - l[k] * z;
        w[k] = ccast<float>(z);
    }
}

// x += Q w (warp per row), FP32 products accumulated then added to the FP64 iterate.
__global__ void __launch_bounds__(256) ref_q_kernel(SolveBufs B, MixBufs M) {
    const EBlk blk = B.tab[blockIdx.y];
    if (M.done[blockIdx.y] || M.fallback[blockIdx.y]) return;
    const int n = blk.n;
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= n) return;
    const c64* Q = M.Q + blk.soff + (long long)row * n;
    const c64* w = M.w32 + blk.off;
    c64 acc = mk<float>(0.f, 0.f);
    for (int j = lane; j < n; j += 32) cmac(acc, Q[j], w[j]);
    acc = warp_sum(acc);
    if (lane == 0) M.x[blk.off + row] = M.x[blk.off + row] + ccast<double>(acc);
}

// Hermitian matvec partials of S x over absolute 64-tiles of the lower triangle (FP64).
__global__ void __launch_bounds__(256) ref_hemv_kernel(SolveBufs B, MixBufs M) {
    __shared__ c128 xs[2][TB];
    __shared__ c128 p2buf[16][TB + 1];
    __shared__ c128 p1s[TB];
    const EBlk blk = B.tab[blockIdx.y];
    if (M.done[blockIdx.y] || M.fallback[blockIdx.y]) return;
    const int n = blk.n;
    const int T = blk.T;
    const long long t = blockIdx.x;
    if (t >= (long long)T * (T + 1) / 2) return;
    long long ii = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
    while (ii * (ii + 1) / 2 > t) --ii;
    const int I = (int)ii, J = (int)(t - ii * (ii + 1) / 2);
    const int tid = threadIdx.x;
    if (tid < 2 * TB) {
        const int which = tid / TB, q = tid % TB;
        const int g = (which == 0 ? I : J) * TB + q;
        xs[which][q] = g < n ? M.x[blk.off + g] : mk<double>(0.0, 0.0);
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
                cmac(p1[a], v, xs[1][c]);
                if (rg > cg) cmacc(p2[bq], v, xs[0][r]);
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
        if (tx == 0) p1s[ty + 16 * a] = p1[a];
    }
#pragma unroll
    for (int bq = 0; bq < 4; ++bq) p2buf[ty][tx + 16 * bq] = p2[bq];
    __syncthreads();
    c128* Y = M.hpart + blk.yoff;
    if (tid < TB) {
        c128 s2 = mk<double>(0.0, 0.0);
#pragma unroll
        for (int k = 0; k < 16; ++k) s2 = s2 + p2buf[k][tid];
        if (I == J) {
            Y[((long long)I * T + I) * TB + tid] = p1s[tid] + s2;
        } else {
            Y[((long long)I * T + J) * TB + tid] = p1s[tid];
            Y[((long long)J * T + I) * TB + tid] = s2;
        }
    }
}

// r = F - (S + shift I) x, FP32 copy of r, ||r||^2 partials.
__global__ void __launch_bounds__(CH) ref_res_kernel(SolveBufs B, MixBufs M, const c128* __restrict__ F, double shift) {
    __shared__ double sh[32];
    const EBlk blk = B.tab[blockIdx.y];
    if (M.done[blockIdx.y] || M.fallback[blockIdx.y]) return;
    const int n = blk.n;
    const int r0 = blockIdx.x * CH;
    if (r0 >= n) return;
    const int r = r0 + threadIdx.x;
    double s = 0.0;
    if (r < n) {
        const int T = blk.T, I = r / TB, rr = r % TB;
        const c128* Y = M.hpart + blk.yoff + (long long)I * T * TB + rr;
        c128 y = mk<double>(0.0, 0.0);
        for (int k = 0; k < T; ++k) y = y + Y[(long long)k * TB];
        const c128 x = M.x[blk.off + r];
        const c128 res = F[blk.off + r] - y - shift * x;
        M.r[blk.off + r] = res;
        M.r32[blk.off + r] = ccast<float>(res);
        s = cabs2(res);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) M.rn[(long long)blockIdx.y * MAXCH + blockIdx.x] = s;
}

__global__ void ref_conv_kernel(SolveBufs B, MixBufs M, int nb, int last, DevStatus* status) {
    const int jb = blockIdx.x * blockDim.x + threadIdx.x;
    if (jb >= nb) return;
    if (M.done[jb] || M.fallback[jb]) return;
    const EBlk blk = B.tab[jb];
    const int nch = (blk.n + CH - 1) / CH;
    double s = 0.0;
    for (int c = 0; c < nch; ++c) s += M.rn[(long long)jb * MAXCH + c];
    if (!(s <= REF_TOL * REF_TOL * M.fn[jb])) {
        if (!isfinite(s)) set_status(status, NQS_ERR_NONFINITE, W_SOLVE, blk.orig);
        else if (last) set_status(status, NQS_ERR_NOT_CONVERGED, W_SOLVE, blk.orig);
        return;
    }
    M.done[jb] = 1;
}

__global__ void ref_out_kernel(SolveBufs B, MixBufs M, double eta, c128* __restrict__ dtheta,
                               int32_t* __restrict__ n_kept) {
    const EBlk blk = B.tab[blockIdx.x];
    for (int k = threadIdx.x; k < blk.n; k += blockDim.x) dtheta[blk.off + k] = (-eta) * M.x[blk.off + k];
    if (threadIdx.x == 0 && n_kept) n_kept[blk.orig] = blk.n;
}

// ------------------------------------------------------------------ host driver
struct Built {
    EBTab tab;
    int nmax;
};

static void build_table(const int64_t* block_off, int nb, Built* bt) {
    EBTab& tab = bt->tab;
    tab.nb = nb;
    int order[MAXB];
    for (int b = 0; b < nb; ++b) order[b] = b;
    for (int x = 1; x < nb; ++x) {  // sort by size, descending: active blocks form a prefix
        const int v = order[x];
        const long long nv = block_off[v + 1] - block_off[v];
        int y = x - 1;
        while (y >= 0 && (block_off[order[y] + 1] - block_off[order[y]]) < nv) {
            order[y + 1] = order[y];
            --y;
        }
        order[y + 1] = v;
    }
    long long soff_of[MAXB + 1];
    soff_of[0] = 0;
    for (int b = 0; b < nb; ++b) {
        const long long n = block_off[b + 1] - block_off[b];
        soff_of[b + 1] = soff_of[b] + n * n;
    }
    long long yacc = 0;
    bt->nmax = 0;
    for (int j = 0; j < nb; ++j) {
        const int b = order[j];
        const int n = (int)(block_off[b + 1] - block_off[b]);
        EBlk& e = tab.b[j];
        e.off = block_off[b];
        e.soff = soff_of[b];
        e.n = n;
        e.T = (n + TB - 1) / TB;
        e.yoff = yacc;
        e.orig = b;
        e.pad = 0;
        yacc += (long long)e.T * e.T * TB;
        bt->nmax = n > bt->nmax ? n : bt->nmax;
    }
}

struct SolveLayoutAll {
    SolveLayout L;
    size_t sf, q, tf, toff, wq, piv, lmul, mx, mr, r32, y32, w32, ypq, hp, rn, fn, done, fb, total;
};

static SolveLayoutAll layout_all(const int64_t* off, int nb) {
    SolveLayoutAll A{};
    A.L = solve_layout(off, nb);
    const long long np = off[nb];
    long long sq = 0, ytot = 0, tfe = 0;
    int nmax = 0;
    for (int b = 0; b < nb; ++b) {
        const long long n = off[b + 1] - off[b];
        sq += n * n;
        const long long T = (n + TB - 1) / TB;
        ytot += T * T * TB;
        tfe += ((n - 1 + QNB - 1) / QNB) * QNB * QNB;
        nmax = n > nmax ? (int)n : nmax;
    }
    const int qch = (nmax + 255) / 256;
    size_t p = A.L.total;
    auto take = [&](size_t bytes) { size_t at = p; p += al(bytes); return at; };
    A.sf = take(8ull * sq);
    A.q = take(8ull * sq);
    A.tf = take(8ull * (tfe > 0 ? tfe : 1));
    A.toff = take(8ull * nb);
    A.wq = take(8ull * QNB * np);
    A.piv = take(8ull * np);
    A.lmul = take(8ull * np);
    A.mx = take(16ull * np);
    A.mr = take(16ull * np);
    A.r32 = take(8ull * np);
    A.y32 = take(8ull * np);
    A.w32 = take(8ull * np);
    A.ypq = take(8ull * qch * np);
    A.hp = take(16ull * ytot);
    A.rn = take(8ull * nb * MAXCH);
    A.fn = take(8ull * nb);
    A.done = take(4ull * nb);
    A.fb = take(4ull * nb);
    A.total = p;
    return A;
}

size_t solve_workspace_bytes(const int64_t* block_off, int nb) { return layout_all(block_off, nb).total; }

__global__ void upload_toff_kernel(const EBTab tab, long long* toff) {
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int j = 0; j < tab.nb; ++j) {
            toff[j] = acc;
            acc += (long long)((tab.b[j].n - 1 + QNB - 1) / QNB) * QNB * QNB;
        }
    }
}

// FP64 path: exact reduction, eigenvalues, LDL^T or QL solve, back-transform.
static int solve_fp64(SolveBufs& B, const EBTab& tab, int nmax, const c128* F, const SolveArgs& a, c128* dtheta,
                      double* evals, int32_t* n_kept, long long np, DevStatus* status, cudaStream_t st) {
    const int nb = tab.nb;
    count_launch();
    init_f_kernel<<<(unsigned)((np + 255) / 256 < 2048 ? (np + 255) / 256 : 2048), 256, 0, st>>>(F, np, B.f);
    TrdBufs<double> T;
    T.tab = B.tab;
    T.A = B.S;
    T.v0 = B.v0;
    T.v1 = B.v1;
    T.w = B.w;
    T.x = B.x;
    T.ypart = B.ypart;
    T.f = B.f;
    T.d = B.d;
    T.e = B.e;
    T.e2 = B.e2;
    T.pnorm = B.pnorm;
    T.tau = B.tau;
    T.pvf = B.pvf;
    T.pxv = B.pxv;
    T.hp = B.hp;
    int rc = trd_reduce<double>(T, tab, st, status);
    if (rc) return rc;
    if (a.ev_trd_done) cudaEventRecord(a.ev_trd_done, st);
    count_launch();
    eig_bounds_kernel<<<(nb + 63) / 64, 64, 0, st>>>(B, nb, a, status);
    if (a.want_evals && evals) {
        count_launch();
        eig_all_kernel<<<dim3((nmax + 127) / 128, nb), 128, 0, st>>>(B, nb, a.shift, B.ev);
    }
    count_launch();
    ldl_solve_kernel<<<(nb + 63) / 64, 64, 0, st>>>(B, nb, a.shift, status);
    if (nmax <= QL_MAXN) {
        const size_t qsm = 2ull * nmax * sizeof(double);
        cudaFuncSetAttribute(ql_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsm);
        // ql_solve_kernel overwrites B.ev (working diagonal) for the blocks it treats,
        // so all-eigenvalue output is copied out before it runs
        if (a.want_evals && evals) cudaMemcpyAsync(evals, B.ev, sizeof(double) * np, cudaMemcpyDeviceToDevice, st);
        count_launch();
        ql_solve_kernel<<<nb, 512, qsm, st>>>(B, nb, a, status);
    } else if (a.want_evals && evals) {
        cudaMemcpyAsync(evals, B.ev, sizeof(double) * np, cudaMemcpyDeviceToDevice, st);
    }
    count_launch();
    back_kernel<<<nb, 512, 0, st>>>(B, nb, a.eta, dtheta, n_kept, status);
    return cudaGetLastError() == cudaSuccess ? NQS_OK : NQS_ERR_CUDA;
}

int launch_block_solve(c128* S, const int64_t* block_off, int nb, const c128* F, const SolveArgs& a, c128* dtheta,
                       double* evals, int32_t* n_kept, void* work, size_t work_bytes, DevStatus* status,
                       cudaStream_t st) {
    if (nb < 1 || nb > MAXB) return NQS_ERR_INVALID_ARG;
    const SolveLayoutAll LA = layout_all(block_off, nb);
    const SolveLayout& L = LA.L;
    if (work_bytes < LA.total) return NQS_ERR_WORKSPACE;
    char* W = static_cast<char*>(work);
    Built bt;
    build_table(block_off, nb, &bt);
    const EBTab& tab = bt.tab;
    const int nmax = bt.nmax;
    if ((nmax + CH - 1) / CH > MAXCH) return NQS_ERR_UNSUPPORTED;
    SolveBufs B;
    B.tab = reinterpret_cast<EBlk*>(W + L.tab);
    B.S = S;
    B.d = reinterpret_cast<double*>(W + L.d);
    B.e = reinterpret_cast<double*>(W + L.e);
    B.e2 = reinterpret_cast<double*>(W + L.e2);
    B.ev = reinterpret_cast<double*>(W + L.ev);
    B.tau = reinterpret_cast<c128*>(W + L.tau);
    B.f = reinterpret_cast<c128*>(W + L.f);
    B.v0 = reinterpret_cast<c128*>(W + L.v0);
    B.v1 = reinterpret_cast<c128*>(W + L.v1);
    B.w = reinterpret_cast<c128*>(W + L.w);
    B.x = reinterpret_cast<c128*>(W + L.x);
    B.z = reinterpret_cast<c128*>(W + L.z);
    B.hp = reinterpret_cast<HouseP*>(W + L.hp);
    B.info = reinterpret_cast<BlkInfo*>(W + L.info);
    B.pnorm = reinterpret_cast<double*>(W + L.pnorm);
    B.pvf = reinterpret_cast<c128*>(W + L.pvf);
    B.pxv = reinterpret_cast<c128*>(W + L.pxv);
    B.ypart = reinterpret_cast<c128*>(W + L.ypart);
    B.zmat = reinterpret_cast<double*>(W + L.zmat);
    const long long np = block_off[nb];
    count_launch();
    upload_tab_kernel<<<1, 256, 0, st>>>(tab, const_cast<EBlk*>(B.tab));
    if (cudaGetLastError() != cudaSuccess) return NQS_ERR_CUDA;
    if (!a.mixed) return solve_fp64(B, tab, nmax, F, a, dtheta, evals, n_kept, np, status, st);

    // ---- mixed precision
    MixBufs M;
    M.tab = B.tab;
    M.S = S;
    M.Sf = reinterpret_cast<c64*>(W + LA.sf);
    M.Q = reinterpret_cast<c64*>(W + LA.q);
    M.Tf = reinterpret_cast<c64*>(W + LA.tf);
    M.toff = reinterpret_cast<long long*>(W + LA.toff);
    M.W = reinterpret_cast<c64*>(W + LA.wq);
    M.d = B.d;
    M.e = B.e;
    M.piv = reinterpret_cast<double*>(W + LA.piv);
    M.lmul = reinterpret_cast<double*>(W + LA.lmul);
    M.x = reinterpret_cast<c128*>(W + LA.mx);
    M.r = reinterpret_cast<c128*>(W + LA.mr);
    M.r32 = reinterpret_cast<c64*>(W + LA.r32);
    M.y32 = reinterpret_cast<c64*>(W + LA.y32);
    M.w32 = reinterpret_cast<c64*>(W + LA.w32);
    M.ypart = reinterpret_cast<c64*>(W + LA.ypq);
    M.hpart = reinterpret_cast<c128*>(W + LA.hp);
    M.rn = reinterpret_cast<double*>(W + LA.rn);
    M.fn = reinterpret_cast<double*>(W + LA.fn);
    M.done = reinterpret_cast<int*>(W + LA.done);
    M.fallback = reinterpret_cast<int*>(W + LA.fb);
    long long sq = 0;
    for (int j = 0; j < nb; ++j) sq += (long long)tab.b[j].n * tab.b[j].n;
    count_launch();
    to_fp32_kernel<<<2048, 256, 0, st>>>(S, sq, M.Sf);
    TrdBufs<float> T;
    T.tab = B.tab;
    T.A = M.Sf;
    T.v0 = reinterpret_cast<c64*>(B.v0);
    T.v1 = reinterpret_cast<c64*>(B.v1);
    T.w = reinterpret_cast<c64*>(B.w);
    T.x = reinterpret_cast<c64*>(B.x);
    T.ypart = reinterpret_cast<c64*>(B.ypart);
    T.f = nullptr;
    T.d = B.d;
    T.e = B.e;
    T.e2 = B.e2;
    T.pnorm = B.pnorm;
    T.tau = B.tau;
    T.pvf = B.pvf;
    T.pxv = B.pxv;
    T.hp = B.hp;
    int rc = trd_reduce<float>(T, tab, st, status);
    if (rc) return rc;
    if (a.ev_trd_done) cudaEventRecord(a.ev_trd_done, st);
    count_launch();
    mix_cert_kernel<<<(nb + 63) / 64, 64, 0, st>>>(B, M, nb, a, status);
    int fb[MAXB];
    if (cudaMemcpyAsync(fb, M.fallback, sizeof(int) * nb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return NQS_ERR_CUDA;
    bool any_fb = false;
    for (int j = 0; j < nb; ++j) any_fb = any_fb || fb[j];
    if (any_fb) {
        // some eigenvalue may be cut: take the exact FP64 path for every block
        return solve_fp64(B, tab, nmax, F, a, dtheta, evals, n_kept, np, status, st);
    }
    if (a.want_evals && evals) {
        count_launch();
        eig_all_kernel<<<dim3((nmax + 127) / 128, nb), 128, 0, st>>>(B, nb, a.shift, evals);
    }
    // explicit Q = H_0 ... H_{n-2} by blocked WY accumulation, last panel first
    count_launch();
    upload_toff_kernel<<<1, 32, 0, st>>>(tab, M.toff);
    const int pmax = (nmax - 1 + QNB - 1) / QNB;
    if (pmax > 0) {
        count_launch();
        qt_factor_kernel<<<dim3(pmax, nb), 256, 0, st>>>(B, M);
    }
    count_launch();
    q_identity_kernel<<<dim3(256, nb), 256, 0, st>>>(B, M);
    for (int p = pmax - 1; p >= 0; --p) {
        const int m = nmax - p * QNB - 1;
        const int tiles = (m + QT - 1) / QT;
        count_launch();
        q_w_kernel<<<dim3(tiles, nb), 256, 0, st>>>(B, M, p);
        count_launch();
        q_update_kernel<<<dim3(tiles, tiles, nb), 256, 0, st>>>(B, M, p);
    }
    if (cudaGetLastError() != cudaSuccess) return NQS_ERR_CUDA;
    // iterative refinement with FP64 residuals
    count_launch();
    ref_init_kernel<<<nb, 256, 0, st>>>(B, M, F);
    const int tq = (nmax + 255) / 256;
    const int T0 = tab.b[0].T;
    for (int it = 0; it < REF_MAXIT; ++it) {
        count_launch();
        ref_qh_kernel<<<dim3(tq, tq, nb), 256, 0, st>>>(B, M, np);
        count_launch();
        ref_tri_kernel<<<(nb + 31) / 32, 32, 0, st>>>(B, M, nb, np);
        count_launch();
        ref_q_kernel<<<dim3((nmax + 7) / 8, nb), 256, 0, st>>>(B, M);
        count_launch();
        ref_hemv_kernel<<<dim3((unsigned)((long long)T0 * (T0 + 1) / 2), nb), 256, 0, st>>>(B, M);
        count_launch();
        ref_res_kernel<<<dim3((nmax + CH - 1) / CH, nb), CH, 0, st>>>(B, M, F, a.shift);
        count_launch();
        ref_conv_kernel<<<(nb + 63) / 64, 64, 0, st>>>(B, M, nb, it == REF_MAXIT - 1, status);
    }
    count_launch();
    ref_out_kernel<<<nb, 256, 0, st>>>(B, M, a.eta, dtheta, n_kept);
    return cudaGetLastError() == cudaSuccess ? NQS_OK : NQS_ERR_CUDA;
}

}  // namespace nqs
