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
#include "eigh.cuh"

namespace nqs {


struct SolveLayout {
    size_t tab, d, e, e2, tau, f, v0, v1, w, x, z, ev, info, bcol, pvf, pxv, ypart, zmat, total;
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
    L.info = take(sizeof(BlkInfo) * nb);
    L.bcol = take(16 * np);
    L.pvf = take(16ull * nb * MAXCH);
    L.pxv = take(16ull * nb * MAXDCH);
    L.ypart = take(16ull * ytot);
    L.zmat = take(8ull * ztot);
    L.total = p;
    return L;
}



__global__ void upload_tab_kernel(const EBTab tab, EBlk* dst) {
    for (int i = threadIdx.x; i < tab.nb; i += blockDim.x) dst[i] = tab.b[i];
}

// Copy F_b into the working vector f (later overwritten by Q^H F_b).
__global__ void init_f_kernel(const c128* __restrict__ F, long long np, c128* __restrict__ f) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x)
        f[p] = F[p];
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

// Gershgorin bounds of T + shift I and the largest e^2, reduced over the CTA.
__device__ void gersh_cta(const double* d, const double* e, const double* e2, int n, double shift, double* lo,
                          double* hi, double* emax) {
    __shared__ double rl[32], rh[32], re[32];
    double gl = 1e300, gu = -1e300, em = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double r = (k > 0 ? fabs(e[k - 1]) : 0.0) + (k < n - 1 ? fabs(e[k]) : 0.0);
        gl = fmin(gl, d[k] + shift - r);
        gu = fmax(gu, d[k] + shift + r);
        if (k + 1 < n) em = fmax(em, e2[k]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        gl = fmin(gl, __shfl_xor_sync(0xffffffffu, gl, o));
        gu = fmax(gu, __shfl_xor_sync(0xffffffffu, gu, o));
        em = fmax(em, __shfl_xor_sync(0xffffffffu, em, o));
    }
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) {
        rl[w] = gl;
        rh[w] = gu;
        re[w] = em;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < nw; ++k) {
            gl = fmin(gl, rl[k]);
            gu = fmax(gu, rh[k]);
            em = fmax(em, re[k]);
        }
        const double span = fmax(fabs(gl), fabs(gu));
        rl[0] = gl - 4.0 * 2.22e-16 * span - 1e-300;
        rh[0] = gu + 4.0 * 2.22e-16 * span + 1e-300;
        re[0] = em;
    }
    __syncthreads();
    *lo = rl[0];
    *hi = rh[0];
    *emax = re[0];
    __syncthreads();
}

// Eigenvalues k0 (first half of the CTA) and k1 (second half) of T + shift I by
// multisection: per round each thread of a half takes the Sturm count at one of its
// interior points, and the bracket of the wanted eigenvalue shrinks (half + 1)-fold.
// Stops when both brackets are narrower than tol (absolute) or after 12 rounds.
__device__ void multisect2(const double* d, const double* e2, int n, double shift, int k0, int k1, double lo0,
                           double hi0, double pivmin, double tol, double* out0, double* out1) {
    __shared__ double blo[2], bhi[2];
    __shared__ int cnt[1024];
    const int half = blockDim.x / 2;
    const int g = threadIdx.x / half, t = threadIdx.x % half;
    const int k = g ? k1 : k0;
    if (threadIdx.x == 0) {
        blo[0] = blo[1] = lo0;
        bhi[0] = bhi[1] = hi0;
    }
    __syncthreads();
    for (int round = 0; round < 12; ++round) {
        const bool open0 = !(bhi[0] - blo[0] <= tol), open1 = !(bhi[1] - blo[1] <= tol);
        if (!open0 && !open1) break;
        const double lo = blo[g], hi = bhi[g];
        const double x = lo + (hi - lo) * (double)(t + 1) / (double)(half + 1);
        cnt[threadIdx.x] = sturm_count(d, e2, n, shift, x, pivmin);
        __syncthreads();
        if (t == 0) {
            double nlo = lo, nhi = hi;
            for (int s2 = 0; s2 < half; ++s2) {
                const double xs = lo + (hi - lo) * (double)(s2 + 1) / (double)(half + 1);
                if (cnt[g * half + s2] <= k) {
                    nlo = xs;
                } else {
                    nhi = xs;
                    break;
                }
            }
            blo[g] = nlo;
            bhi[g] = nhi;
        }
        __syncthreads();
    }
    *out0 = 0.5 * (blo[0] + bhi[0]);
    *out1 = 0.5 * (blo[1] + bhi[1]);
    __syncthreads();
}

// One CTA per block: sigma_max (multisection to full precision), threshold, number dropped.
__global__ void __launch_bounds__(256) eig_bounds_kernel(SolveBufs B, int nb, SolveArgs a, DevStatus* status) {
    const int j = blockIdx.x;
    const EBlk blk = B.tab[j];
    const int n = blk.n;
    const double* d = B.d + blk.off;
    const double* e = B.e + blk.off;
    const double* e2 = B.e2 + blk.off;
    double lo, hi, emax;
    gersh_cta(d, e, e2, n, a.shift, &lo, &hi, &emax);
    const double pivmin = 1e-290 * fmax(1.0, emax);
    double smax, smax2;
    multisect2(d, e2, n, a.shift, n - 1, n - 1, lo, hi, pivmin, 4.0 * 2.22e-16 * fmax(fabs(lo), fabs(hi)), &smax,
               &smax2);
    if (threadIdx.x != 0) return;
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
    if (B.info[blockIdx.x].n_dropped == 0 && !a.want_vectors) return;
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
    const int maxit = a.ql_maxit;
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
    if (threadIdx.x == 0) {
        double mx = -1e300;
        for (int k = 0; k < n; ++k) mx = fmax(mx, dd[k]);
        const double thr = a.cutoff_mode == 0 ? a.cutoff * mx : a.cutoff;
        int kept = 0;
        for (int k = 0; k < n; ++k) kept += dd[k] > thr;
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

__global__ void to_fp32_kernel(const c128* __restrict__ S, long long n, c64* __restrict__ Sf) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        Sf[i] = ccast<float>(S[i]);
}

// Sturm count in FP32 on (d + shift, e^2) stored as floats: the number of eigenvalues of
// T + shift I below x. The LDL^T pivot recurrence is backward stable, so the count is exact for
// a tridiagonal within a few FP32 ulps of the stored one.
__device__ __forceinline__ int sturm_count_f(const float* __restrict__ ds, const float* __restrict__ e2, int n,
                                             float x, float pivmin) {
    int cnt = 0;
    float q = ds[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += q < 0.f;
    for (int k = 1; k < n; ++k) {
        q = (ds[k] - x) - __fdividef(e2[k - 1], q);
        if (fabsf(q) < pivmin) q = -pivmin;
        cnt += q < 0.f;
    }
    return cnt;
}

// multisect2 with FP32 Sturm counts (brackets kept in FP64)
__device__ void multisect2_f(const float* ds, const float* e2, int n, int k0, int k1, double lo0, double hi0,
                             float pivmin, double tol, double* out0, double* out1) {
    __shared__ double blo[2], bhi[2];
    __shared__ int cnt[1024];
    const int half = blockDim.x / 2;
    const int g = threadIdx.x / half, t = threadIdx.x % half;
    const int k = g ? k1 : k0;
    if (threadIdx.x == 0) {
        blo[0] = blo[1] = lo0;
        bhi[0] = bhi[1] = hi0;
    }
    __syncthreads();
    for (int round = 0; round < 12; ++round) {
        const bool open0 = !(bhi[0] - blo[0] <= tol), open1 = !(bhi[1] - blo[1] <= tol);
        if (!open0 && !open1) break;
        const double lo = blo[g], hi = bhi[g];
        const double x = lo + (hi - lo) * (double)(t + 1) / (double)(half + 1);
        cnt[threadIdx.x] = sturm_count_f(ds, e2, n, (float)x, pivmin);
        __syncthreads();
        if (t == 0) {
            double nlo = lo, nhi = hi;
            for (int s2 = 0; s2 < half; ++s2) {
                const double xs = lo + (hi - lo) * (double)(s2 + 1) / (double)(half + 1);
                if (cnt[g * half + s2] <= k) {
                    nlo = xs;
                } else {
                    nhi = xs;
                    break;
                }
            }
            blo[g] = nlo;
            bhi[g] = nhi;
        }
        __syncthreads();
    }
    *out0 = 0.5 * (blo[0] + bhi[0]);
    *out1 = 0.5 * (blo[1] + bhi[1]);
    __syncthreads();
}

// One CTA per block: FP32-based bounds; a block needs the FP64 path when an eigenvalue
// might fall on the dropped side of the cutoff within the FP32 error. The bounds need
// only ~1e-10 relative accuracy (the certificate allows 4e-5).
__global__ void __launch_bounds__(256) mix_cert_kernel(SolveBufs B, MixBufs M, int nb, SolveArgs a, DevStatus* status) {
    const int j = blockIdx.x;
    const EBlk blk = B.tab[j];
    const int n = blk.n;
    const double* d = M.d + blk.off;
    const double* e = M.e + blk.off;
    const double* e2 = B.e2 + blk.off;
    double lo, hi, emax;
    gersh_cta(d, e, e2, n, a.shift, &lo, &hi, &emax);
    const double pivmin = 1e-290 * fmax(1.0, emax);
    float* ds = M.ds32 + blk.off;
    float* ef = M.e232 + blk.off;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        ds[k] = (float)(d[k] + a.shift);
        ef[k] = k + 1 < n ? (float)e2[k] : 0.f;
    }
    __syncthreads();
    // the certificate allows 4e-5 sigma_max: FP32 counts to ~1e-6 of the Gershgorin span suffice
    const float pivf = fmaxf(1e-30f, 1e-30f * (float)emax);
    double smax, smin;
    multisect2_f(ds, ef, n, n - 1, 0, lo, hi, pivf, 1e-6 * fmax(fabs(lo), fabs(hi)), &smax, &smin);
    (void)pivmin;
    if (threadIdx.x != 0) return;
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

__global__ void not_done_status_kernel(const int* __restrict__ done, int nb, DevStatus* status) {
    int any = 0;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) any |= !done[j];
    if (__any_sync(0xffffffffu, any) && threadIdx.x == 0) set_status(status, NQS_ERR_RETRY, W_SOLVE, -2);
}

__global__ void retry_status_kernel(const int* __restrict__ fallback, int nb, DevStatus* status) {
    int any = 0;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) any |= fallback[j];
    if (__any_sync(0xffffffffu, any) && threadIdx.x == 0) set_status(status, NQS_ERR_RETRY, W_SOLVE, -1);
}

// (h, l) += a b for FP32 a, b: exact product by FMA, TwoSum into the high word, errors to
// the low word (double-float accumulation).
__device__ __forceinline__ void df_acc(float& h, float& l, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);
    const float s = __fadd_rn(h, p);
    const float bb = __fsub_rn(s, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    h = s;
    l = __fadd_rn(l, __fadd_rn(e, pe));
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
    // G = V^H V over rows r in [i0+1, n); V[r][j] = A[(i0+j) n + r] for r >= i0+j+1, else 0.
    // The products of the FP32 reflector entries are made exact with an FMA and summed in
    // double-float (hi + lo) on the FP32 units, about 2^-46 relative.
    const int npairs = nbp * (nbp + 1) / 2;
    for (int idx = threadIdx.x; idx < npairs; idx += blockDim.x) {
        int b = (int)((sqrtf(8.f * (float)idx + 1.f) - 1.f) * 0.5f);  // pair (a, b), a <= b
        while ((b + 1) * (b + 2) / 2 <= idx) ++b;
        while (b * (b + 1) / 2 > idx) --b;
        const int a = idx - b * (b + 1) / 2;
        const int r0 = i0 + b + 1;  // both vectors nonzero from max(a, b) + i0 + 1
        const c64* va = A + (long long)(i0 + a) * n;
        const c64* vb = A + (long long)(i0 + b) * n;
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
#pragma unroll 4
        for (int r = r0; r < n; ++r) {
            const c64 x = va[r], y = vb[r];  // conj(x) y
            df_acc(rh, rl, x.re, y.re);
            df_acc(rh, rl, x.im, y.im);
            df_acc(ih, il, x.re, y.im);
            df_acc(ih, il, -x.im, y.re);
        }
        G[a][b] = mk<double>((double)rh + (double)rl, (double)ih + (double)il);
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
    size_t sf, tf, toff, pdot, bar, piv, lmul, ds32, e232, mx, mr, r32, y32, w32, hpart, rn, fn, done, fb, total;
};

static SolveLayoutAll layout_all(const int64_t* off, int nb) {
    SolveLayoutAll A{};
    A.L = solve_layout(off, nb);
    const long long np = off[nb];
    long long sq = 0, ytot = 0, tfe = 0, totch = 0;
    for (int b = 0; b < nb; ++b) {
        const long long n = off[b + 1] - off[b];
        sq += n * n;
        const long long T = (n + TB - 1) / TB;
        ytot += T * T * TB;
        tfe += ((n - 1 + QNB - 1) / QNB) * QNB * QNB;
        totch += (n + CH - 1) / CH;
    }
    size_t p = A.L.total;
    auto take = [&](size_t bytes) { size_t at = p; p += al(bytes); return at; };
    // the FP32 copy of the eigen path and the Cholesky path's buffers share one region: the
    // eigen path runs only after the Cholesky path has finished (host-synchronised fallback)
    const size_t chol = chol_workspace_bytes(off, nb);
    A.sf = take(8ull * sq > chol ? 8ull * sq : chol);
    A.tf = take(8ull * (tfe > 0 ? tfe : 1));
    A.toff = take(8ull * nb);
    A.pdot = take(8ull * 2 * totch * QNB);
    A.bar = take(64);
    A.piv = take(8ull * np);
    A.ds32 = take(4ull * np);
    A.e232 = take(4ull * np);
    A.lmul = take(8ull * np);
    A.mx = take(16ull * np);
    A.mr = take(16ull * np);
    A.r32 = take(8ull * np);
    A.y32 = take(8ull * np);
    A.w32 = take(8ull * np);
    A.hpart = take(16ull * ytot);
    A.rn = take(8ull * nb * MAXDCH);
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
    T.bcol = reinterpret_cast<decltype(T.bcol)>(B.bcol);
    T.tau = B.tau;
    T.pvf = B.pvf;
    T.pxv = B.pxv;
    if (a.ev_trd_start) cudaEventRecord(a.ev_trd_start, st);
    int rc = launch_trd_persist<double>(T, tab, B.bar, status, st);
    if (rc) return rc;
    if (a.ev_trd_done) cudaEventRecord(a.ev_trd_done, st);
    count_launch();
    eig_bounds_kernel<<<nb, 256, 0, st>>>(B, nb, a, status);
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

// U[i][:] = Q z_i for every tridiagonal eigenvector z_i (row i of the QL's Zt) of block 0:
// the reflectors H_k = I - tau_k v_k v_k^H applied for k = n-2 .. 0 (eigenvector-major output).
__global__ void __launch_bounds__(256) eigvec_back_kernel(SolveBufs B, c128* __restrict__ U) {
    __shared__ double sh[32];
    const EBlk blk = B.tab[0];
    const int n = blk.n;
    const c128* A = B.S + blk.soff;
    const double* zt = B.zmat + blk.soff + (long long)blockIdx.x * n;
    c128* u = U + (long long)blockIdx.x * n;
    for (int r = threadIdx.x; r < n; r += blockDim.x) u[r] = mk<double>(zt[r], 0.0);
    __syncthreads();
    for (int k = n - 2; k >= 0; --k) {
        const c128 tau = B.tau[blk.off + k];
        if (tau.re == 0.0 && tau.im == 0.0) continue;
        const c128* v = A + (long long)k * n;  // v[r] for r >= k+1
        c128 dot = mk<double>(0.0, 0.0);
        for (int r = k + 1 + threadIdx.x; r < n; r += blockDim.x) cmacc(dot, v[r], u[r]);
        dot.re = block_sum(dot.re, sh);
        dot.im = block_sum(dot.im, sh);
        const c128 g = tau * dot;
        for (int r = k + 1 + threadIdx.x; r < n; r += blockDim.x) u[r] = u[r] - g * v[r];
        __syncthreads();
    }
}

__global__ void zero_c128_kernel(c128* __restrict__ p, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = mk<double>(0.0, 0.0);
}

size_t eig_vectors_workspace_bytes(long long n) {
    const int64_t off[2] = {0, n};
    return solve_workspace_bytes(off, 1) + 2 * al(16ull * n);
}

int launch_eig_vectors(c128* S, long long n, double shift, double* sig, double* evals_asc, c128* U, void* work,
                       size_t work_bytes, DevStatus* status, cudaStream_t st) {
    if (n < 1 || n > QL_MAXN) return NQS_ERR_UNSUPPORTED;
    const int64_t off[2] = {0, n};
    const SolveLayoutAll LA = layout_all(off, 1);
    if (work_bytes < eig_vectors_workspace_bytes(n)) return NQS_ERR_WORKSPACE;
    char* W = static_cast<char*>(work);
    c128* F0 = reinterpret_cast<c128*>(W + LA.total);
    c128* dth = reinterpret_cast<c128*>(W + LA.total + al(16ull * n));
    count_launch();
    zero_c128_kernel<<<64, 256, 0, st>>>(F0, n);
    SolveArgs a{};
    a.shift = shift;
    a.cutoff = 0.0;  // every eigenvalue kept here: the diagnostics apply their own cutoff
    a.eta = 1.0;
    a.cutoff_mode = 0;
    a.want_evals = true;
    a.ql_maxit = limits().ql_maxit;
    a.want_vectors = true;
    Built bt;
    build_table(off, 1, &bt);
    SolveBufs B;
    const SolveLayout& L = LA.L;
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
    B.info = reinterpret_cast<BlkInfo*>(W + L.info);
    B.bcol = reinterpret_cast<c128*>(W + L.bcol);
    B.pvf = reinterpret_cast<c128*>(W + L.pvf);
    B.pxv = reinterpret_cast<c128*>(W + L.pxv);
    B.ypart = reinterpret_cast<c128*>(W + L.ypart);
    B.zmat = reinterpret_cast<double*>(W + L.zmat);
    B.bar = reinterpret_cast<unsigned*>(W + LA.bar);
    count_launch();
    upload_tab_kernel<<<1, 256, 0, st>>>(bt.tab, const_cast<EBlk*>(B.tab));
    if (cudaGetLastError() != cudaSuccess) return NQS_ERR_CUDA;
    int rc = solve_fp64(B, bt.tab, bt.nmax, F0, a, dth, evals_asc, nullptr, n, status, st);
    if (rc) return rc;
    count_launch();
    eigvec_back_kernel<<<(unsigned)n, 256, 0, st>>>(B, U);
    if (cudaMemcpyAsync(sig, B.ev, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return NQS_ERR_CUDA;
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
    B.info = reinterpret_cast<BlkInfo*>(W + L.info);
    B.bcol = reinterpret_cast<c128*>(W + L.bcol);
    B.pvf = reinterpret_cast<c128*>(W + L.pvf);
    B.pxv = reinterpret_cast<c128*>(W + L.pxv);
    B.ypart = reinterpret_cast<c128*>(W + L.ypart);
    B.zmat = reinterpret_cast<double*>(W + L.zmat);
    B.bar = reinterpret_cast<unsigned*>(W + LA.bar);
    const long long np = block_off[nb];
    count_launch();
    upload_tab_kernel<<<1, 256, 0, st>>>(tab, const_cast<EBlk*>(B.tab));
    if (cudaGetLastError() != cudaSuccess) return NQS_ERR_CUDA;
    if (!a.mixed) return solve_fp64(B, tab, nmax, F, a, dtheta, evals, n_kept, np, status, st);

    // ---- Gram-matrix blocks, eigenvalues not requested: certified Cholesky + refinement
    if (a.psd && !(a.want_evals && evals) && chol_applicable(block_off, nb)) {
        bool ok = false;
        const size_t cb = chol_workspace_bytes(block_off, nb);
        const int rc = launch_chol_solve(S, block_off, nb, F, a, dtheta, n_kept, W + LA.sf, cb, status, st, &ok);
        if (rc) return rc;
        if (ok) return NQS_OK;
        // some block not certified, not factored or not converged: eigen-decomposition path
    }

    // ---- mixed precision
    MixBufs M;
    M.tab = B.tab;
    M.S = S;
    M.Sf = reinterpret_cast<c64*>(W + LA.sf);
    M.Tf = reinterpret_cast<c64*>(W + LA.tf);
    M.toff = reinterpret_cast<long long*>(W + LA.toff);
    M.pdot = reinterpret_cast<c64*>(W + LA.pdot);
    M.d = B.d;
    M.e = B.e;
    M.piv = reinterpret_cast<double*>(W + LA.piv);
    M.ds32 = reinterpret_cast<float*>(W + LA.ds32);
    M.e232 = reinterpret_cast<float*>(W + LA.e232);
    M.lmul = reinterpret_cast<double*>(W + LA.lmul);
    M.x = reinterpret_cast<c128*>(W + LA.mx);
    M.r = reinterpret_cast<c128*>(W + LA.mr);
    M.r32 = reinterpret_cast<c64*>(W + LA.r32);
    M.y32 = reinterpret_cast<c64*>(W + LA.y32);
    M.w32 = reinterpret_cast<c64*>(W + LA.w32);
    M.hpart = reinterpret_cast<c128*>(W + LA.hpart);
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
    T.bcol = reinterpret_cast<decltype(T.bcol)>(B.bcol);
    T.tau = B.tau;
    T.pvf = B.pvf;
    T.pxv = B.pxv;
    if (a.ev_trd_start) cudaEventRecord(a.ev_trd_start, st);
    int rc = launch_trd_persist<float>(T, tab, B.bar, status, st);
    if (rc) return rc;
    if (a.ev_trd_done) cudaEventRecord(a.ev_trd_done, st);
    count_launch();
    mix_cert_kernel<<<nb, 256, 0, st>>>(B, M, nb, a, status);
    if (a.no_host_sync) {
        // capturable form: a failed certificate is reported, the caller retakes the step
        count_launch();
        retry_status_kernel<<<1, 32, 0, st>>>(M.fallback, nb, status);
    } else {
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
    }
    if (a.want_evals && evals) {
        count_launch();
        eig_all_kernel<<<dim3((nmax + 127) / 128, nb), 128, 0, st>>>(B, nb, a.shift, evals);
    }
    // T factors of the reflector panels (blocked WY form of Q), then the refinement
    count_launch();
    upload_toff_kernel<<<1, 32, 0, st>>>(tab, M.toff);
    const int pmax = (nmax - 1 + QNB - 1) / QNB;
    if (pmax > 0) {
        count_launch();
        qt_factor_kernel<<<dim3(pmax, nb), 256, 0, st>>>(B, M);
    }
    if (cudaGetLastError() != cudaSuccess) return NQS_ERR_CUDA;
    rc = launch_refine_persist(B, M, tab, F, a.shift, B.bar, status, st);
    if (rc) return rc;
    count_launch();
    ref_out_kernel<<<nb, 256, 0, st>>>(B, M, a.eta, dtheta, n_kept);
    if (cudaGetLastError() != cudaSuccess) return NQS_ERR_CUDA;
    // a block whose refinement did not converge: the FP64 path for every block
    if (a.no_host_sync) {
        count_launch();
        not_done_status_kernel<<<1, 32, 0, st>>>(M.done, nb, status);
        return cudaGetLastError() == cudaSuccess ? NQS_OK : NQS_ERR_CUDA;
    }
    int dn[MAXB];
    if (cudaMemcpyAsync(dn, M.done, sizeof(int) * nb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return NQS_ERR_CUDA;
    for (int j = 0; j < nb; ++j)
        if (!dn[j]) return solve_fp64(B, tab, nmax, F, a, dtheta, evals, n_kept, np, status, st);
    return NQS_OK;
}

}  // namespace nqs
