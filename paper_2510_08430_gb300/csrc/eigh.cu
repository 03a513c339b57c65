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

size_t solve_workspace_bytes(const int64_t* block_off, int nb) { return solve_layout(block_off, nb).total; }

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
    long long* zoff;  // unused placeholder
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
__global__ void __launch_bounds__(CH) trd_col_kernel(SolveBufs B, int i, const c128* __restrict__ vprev,
                                                     DevStatus* status) {
    __shared__ double sh[32];
    const EBlk blk = B.tab[blockIdx.y];
    const int n = blk.n;
    if (i > n - 1) return;
    const long long r = (long long)i + (long long)blockIdx.x * CH + threadIdx.x;
    if ((long long)i + (long long)blockIdx.x * CH >= n) return;  // whole CTA past the end
    c128* A = B.S + blk.soff;
    double nrm = 0.0;
    if (r < n) {
        c128 a = A[r * n + i];
        if (i >= 1) {
            const c128* vp = vprev + blk.off;
            const c128* wp = B.w + blk.off;
            const c128 vpi = vp[i], wpi = wp[i];
            const c128 vr = vp[r], wr = B.w[blk.off + r];
            a = a - vr * cconj(wpi) - wr * cconj(vpi);
        }
        if (r == i) a.im = 0.0;
        A[r * n + i] = a;
        if (r >= i + 2) nrm = cabs2(a);
    }
    nrm = block_sum(nrm, sh);
    if (threadIdx.x == 0) B.pnorm[(long long)blockIdx.y * MAXCH + blockIdx.x] = nrm;
}

// K2: Householder reflector of column i (LAPACK-style: beta real, H^H [alpha; x] = [beta; 0]).
__global__ void trd_house_kernel(SolveBufs B, int i, int nch, DevStatus* status) {
    const EBlk blk = B.tab[blockIdx.x];
    const int n = blk.n;
    if (i > n - 1) return;
    const c128* A = B.S + blk.soff;
    const int lane = threadIdx.x;
    const int my_nch = (n - i + CH - 1) / CH;  // chunks written by trd_col_kernel for this block
    (void)nch;
    double xn = 0.0;
    for (int c = lane; c < my_nch; c += 32) xn += B.pnorm[(long long)blockIdx.x * MAXCH + c];
    xn = warp_sum(xn);
    if (lane != 0) return;
    B.d[blk.off + i] = A[(long long)i * n + i].re;
    if (i > n - 2) return;
    const c128 alpha = A[(long long)(i + 1) * n + i];
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
__global__ void __launch_bounds__(CH) trd_v_kernel(SolveBufs B, int i, c128* __restrict__ vcur) {
    __shared__ double sh[32];
    const EBlk blk = B.tab[blockIdx.y];
    const int n = blk.n;
    if (i > n - 2) return;
    const long long base = (long long)i + 1 + (long long)blockIdx.x * CH;
    if (base >= n) return;
    const long long r = base + threadIdx.x;
    c128* A = B.S + blk.soff;
    const HouseP h = B.hp[blockIdx.y];
    c128 vf = mk<double>(0.0, 0.0);
    if (r < n) {
        const c128 v = (r == i + 1) ? mk<double>(1.0, 0.0) : A[r * n + i] * h.scale;
        vcur[blk.off + r] = v;
        A[(long long)i * n + r] = v;
        cmacc(vf, v, B.f[blk.off + r]);
    }
    vf.re = block_sum(vf.re, sh);
    vf.im = block_sum(vf.im, sh);
    if (threadIdx.x == 0) B.pvf[(long long)blockIdx.y * MAXCH + blockIdx.x] = vf;
}

// K4: on the trailing region [i+1, n)^2 (lower triangle, absolute 64-tiles):
//   A -= v_{i-1} w_{i-1}^H + w_{i-1} v_{i-1}^H      (pending update, if i >= 1)
//   y  = A v_i                                        (Hermitian matvec partials)
__global__ void __launch_bounds__(256) trd_fused_kernel(SolveBufs B, int i, const c128* __restrict__ vprev,
                                                         const c128* __restrict__ vcur) {
    __shared__ c128 sv[2][TB], svp[2][TB], swp[2][TB];
    __shared__ c128 p2buf[16][TB + 1];
    __shared__ c128 p1s[TB];
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
    if (tid < 2 * TB) {
        const int which = tid / TB, q = tid % TB;
        const int g = (which == 0 ? I : J) * TB + q;
        c128 vv = mk<double>(0.0, 0.0), vp = vv, wp = vv;
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
    c128* A = B.S + blk.soff;
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
            if (rg < n && cg < n && cg >= R0 && rg >= cg) {
                const long long idx = (long long)rg * n + cg;
                c128 x = A[idx];
                if (pend) {
                    x = x - svp[0][r] * cconj(swp[1][c]) - swp[0][r] * cconj(svp[1][c]);
                    if (rg == cg) x.im = 0.0;
                    A[idx] = x;
                }
                cmac(p1[a], x, sv[1][c]);
                if (rg > cg) cmacc(p2[bq], x, sv[0][r]);
            }
        }
    }
    // p1: reduce over the 16 tx lanes of each half-warp
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
    c128* Y = B.ypart + blk.yoff;
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

// K5: y = sum of matvec partials, x = tau y, partial x^H v.
__global__ void __launch_bounds__(CH) trd_w1_kernel(SolveBufs B, int i, const c128* __restrict__ vcur) {
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
        const c128* Y = B.ypart + blk.yoff + (long long)I * T * TB + rr;
        c128 y = mk<double>(0.0, 0.0);
        for (int s = J0; s < T; ++s) y = y + Y[(long long)s * TB];
        const c128 x = tau * y;
        B.x[blk.off + r] = x;
        cmacc(xv, x, vcur[blk.off + r]);
    }
    xv.re = block_sum(xv.re, sh);
    xv.im = block_sum(xv.im, sh);
    if (threadIdx.x == 0) B.pxv[(long long)blockIdx.y * MAXCH + blockIdx.x] = xv;
}

// K6: w = x - 0.5 tau (x^H v) v; f <- H^H f = f - conj(tau) v (v^H f).
__global__ void __launch_bounds__(CH) trd_w2_kernel(SolveBufs B, int i, int nch, const c128* __restrict__ vcur) {
    __shared__ c128 red[2];
    const EBlk blk = B.tab[blockIdx.y];
    const int n = blk.n;
    if (i > n - 2) return;
    const long long base = (long long)i + 1 + (long long)blockIdx.x * CH;
    if (base >= n) return;
    if (threadIdx.x < 32) {
        const int my_nch = (n - i - 1 + CH - 1) / CH;  // chunks of rows [i+1, n)
        (void)nch;
        c128 a = mk<double>(0.0, 0.0), b = a;
        for (int c = threadIdx.x; c < my_nch; c += 32) {
            a = a + B.pxv[(long long)blockIdx.y * MAXCH + c];
            b = b + B.pvf[(long long)blockIdx.y * MAXCH + c];
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
    const c128 v = vcur[blk.off + r];
    B.w[blk.off + r] = B.x[blk.off + r] + alpha * v;
    const c128 g = cconj(tau) * red[1];
    B.f[blk.off + r] = B.f[blk.off + r] - g * v;
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

// ------------------------------------------------------------------ host driver
int launch_block_solve(c128* S, const int64_t* block_off, int nb, const c128* F, const SolveArgs& a,
                       c128* dtheta, double* evals, int32_t* n_kept, void* work, size_t work_bytes,
                       DevStatus* status, cudaStream_t st) {
    if (nb < 1 || nb > MAXB) return NQS_ERR_INVALID_ARG;
    const SolveLayout L = solve_layout(block_off, nb);
    if (work_bytes < L.total) return NQS_ERR_WORKSPACE;
    char* W = static_cast<char*>(work);
    EBTab tab;
    tab.nb = nb;
    // sort blocks by size (descending) so that active blocks form a prefix
    int order[MAXB];
    for (int b = 0; b < nb; ++b) order[b] = b;
    for (int x = 1; x < nb; ++x) {
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
    int nmax = 0;
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
        nmax = n > nmax ? n : nmax;
    }
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
    B.zoff = nullptr;
    const long long np = block_off[nb];
    count_launch();
    upload_tab_kernel<<<1, 256, 0, st>>>(tab, const_cast<EBlk*>(B.tab));
    count_launch();
    init_f_kernel<<<(unsigned)((np + 255) / 256 < 2048 ? (np + 255) / 256 : 2048), 256, 0, st>>>(F, np, B.f);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return NQS_ERR_CUDA;
    // sizes of sorted blocks for the per-step active counts
    int ns_sorted[MAXB];
    for (int j = 0; j < nb; ++j) ns_sorted[j] = tab.b[j].n;
    for (int i = 0; i < nmax; ++i) {
        int act1 = 0, act2 = 0;  // blocks with n-1 >= i, with n-2 >= i
        while (act1 < nb && ns_sorted[act1] - 1 >= i) ++act1;
        while (act2 < nb && ns_sorted[act2] - 2 >= i) ++act2;
        c128* vcur = (i & 1) ? B.v1 : B.v0;
        c128* vprev = (i & 1) ? B.v0 : B.v1;
        const int nch1 = (nmax - i + CH - 1) / CH;
        count_launch();
        trd_col_kernel<<<dim3(nch1, act1), CH, 0, st>>>(B, i, vprev, status);
        count_launch();
        trd_house_kernel<<<act1, 32, 0, st>>>(B, i, nch1, status);
        if (act2 > 0) {
            const int nch2 = (nmax - i - 1 + CH - 1) / CH;
            count_launch();
            trd_v_kernel<<<dim3(nch2, act2), CH, 0, st>>>(B, i, vcur);
            const int T0 = tab.b[0].T, J0 = (i + 1) / TB;
            const long long cnt = (long long)(T0 - J0) * (T0 - J0 + 1) / 2;
            count_launch();
            trd_fused_kernel<<<dim3((unsigned)cnt, act2), 256, 0, st>>>(B, i, vprev, vcur);
            count_launch();
            trd_w1_kernel<<<dim3(nch2, act2), CH, 0, st>>>(B, i, vcur);
            count_launch();
            trd_w2_kernel<<<dim3(nch2, act2), CH, 0, st>>>(B, i, nch2, vcur);
        }
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return NQS_ERR_CUDA;
    }
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
        if (a.want_evals && evals) {
            cudaMemcpyAsync(evals, B.ev, sizeof(double) * np, cudaMemcpyDeviceToDevice, st);
        }
        count_launch();
        ql_solve_kernel<<<nb, 512, qsm, st>>>(B, nb, a, status);
    } else if (a.want_evals && evals) {
        cudaMemcpyAsync(evals, B.ev, sizeof(double) * np, cudaMemcpyDeviceToDevice, st);
    }
    count_launch();
    back_kernel<<<nb, 512, 0, st>>>(B, nb, a.eta, dtheta, n_kept, status);
    ce = cudaGetLastError();
    return ce == cudaSuccess ? NQS_OK : NQS_ERR_CUDA;
}

}  // namespace nqs
