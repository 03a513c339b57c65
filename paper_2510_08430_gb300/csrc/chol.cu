// Cholesky path of the per-block shifted solve (Sec. 2, block-layer paragraph:
// dtheta_b = -eta pinv(S_b + lambda I) F_b) for blocks that are Gram matrices.
//
// When no eigenvalue of S~_b = S_b + lambda I falls below the cutoff, the pseudo-inverse is
// the inverse and the update is the solution of the Hermitian positive-definite system
// S~_b x = F_b. The cutoff is certified without an eigen-decomposition:
//   sigma_max(S~_b) <= ||S_b||_F + lambda                     (any Hermitian matrix)
//   sigma_min(S~_b) >= lambda - 1e-6 ||S_b||_F                 (S_b a Gram matrix up to rounding)
//   keep-all  <=>  lower bound > cutoff * upper bound (relative mode) or > cutoff (absolute).
// Certified blocks are solved by mixed-precision iterative refinement:
//   S~_b ~= L L^H in FP32 (right-looking, 64 x 64 tiles):
//     potrf  diagonal tile: unblocked Cholesky and the inverse of L_kk (one CTA per block),
//     trsm   panel tiles  : L_ik = A_ik L_kk^-H, a tile product with the stored inverse,
//     herk   trailing     : A_ij -= L_ik L_jk^H for k < j <= i (SIMT FP32 tile products);
//   x_0 = 0;  r = F - S~ x (FP64, from the FP64 S_b);  x += L^-H L^-1 r  until
//   ||r|| <= 1e-14 ||F||. The triangular solves run as a wavefront over tile rows: a tile row
//   waits (bounded) for the rows it depends on, then applies its off-diagonal tiles and the
//   stored diagonal inverse. All sweeps run in one cooperative launch.
// Any block whose certificate fails, whose FP32 factor meets a non-positive pivot, or whose
// refinement does not converge is flagged; the caller then solves every block by the
// eigen-decomposition path instead (or, under stream capture, reports NQS_ERR_RETRY).
#include <new>
#include "eigh.cuh"

namespace nqs {
namespace {

constexpr int CT = 64;                 // tile edge
constexpr int CTE = CT * CT;           // elements per tile
constexpr int CP = 256;                // threads per CTA
constexpr int LDT = CT + 1;            // padded leading dimension of shared tiles
constexpr int CHOL_MAXT = 1024;        // tiles per block edge (n <= 65536)
constexpr double CHOL_TOL = 1e-14;     // default of ||r|| <= tol ||F|| (SolveArgs::ref_tol), or
constexpr double CHOL_FLOOR = 1e-12;   // ||r|| <= CHOL_FLOOR ||F|| once ||r|| stops contracting (the
                                       // FP64 residual's rounding floor, ~n u ||S~|| ||x||)
constexpr double PSD_MARGIN = 1e-6;    // rounding of a Gram matrix's eigenvalues, relative to ||S||

enum : int { CF_CERT = 1, CF_PIVOT = 2, CF_CONV = 4, CF_NONFINITE = 8 };

struct CBlk {
    long long off;    // offset of the block in length-n_p arrays (F, dtheta)
    long long soff;   // offset of S_b in the packed FP64 S (n x n, row-major, lower used)
    long long toff;   // first lower tile of the block in the tiled factor
    long long doff;   // first tile row of the block (diagonal inverses, padded vectors)
    long long poff;   // first residual partial vector of the block (T x T vectors of CT)
    int n, T, orig, pad;
};
struct CTab {
    int nb, Tmax;
    long long tiles, rows, parts;   // totals: lower tiles, tile rows, partial vectors
    CBlk b[MAXB];
};

struct CBufs {
    const CBlk* tab;
    const long long* pref;   // [2][Tmax][nb + 1]: per panel, prefix of trsm / herk units
    c64* L;                  // lower tiles, tile (i, j) of block b at toff + i(i+1)/2 + j
    c64* Dinv;               // inverse of each diagonal tile L_kk (lower), at doff + k
    double* fro;             // per lower tile: its share of ||S_b||_F^2
    int* flags;              // per block (table order): CF_* bits
    c128* P;                 // residual partials: P[poff + i T + j][CT] = (S~ x) part of row tile i
    c128 *x, *r;             // FP64 iterate and residual, padded (doff * CT)
    c64 *r32, *y, *z;        // FP32 residual, forward and backward solutions
    double* rn;              // per tile row ||r||^2
    int* done;               // per block
    unsigned *fflag, *bflag; // per tile row: sweep + 1 once y (forward) / z (backward) is written
    unsigned* bar;           // grid-barrier words
};

__device__ __forceinline__ unsigned long long gtime_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Block of unit u: the last b with pref[b] <= u (pref[0] = 0, non-decreasing).
__device__ __forceinline__ int find_block(const long long* pref, int nb, long long u) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pref[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// (i, j), i >= j, of lower-triangle index t = i (i + 1) / 2 + j.
__device__ __forceinline__ void tri_ij(long long t, int* I, int* J) {
    long long i = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    *I = (int)i;
    *J = (int)(t - i * (i + 1) / 2);
}

__device__ __forceinline__ long long tile_at(const CBlk& b, int i, int j) {
    return b.toff + (long long)i * (i + 1) / 2 + j;
}

// ------------------------------------------------------------------ set-up
__global__ void chol_upload_kernel(const CTab tab, CBlk* dst) {
    for (int i = threadIdx.x; i < tab.nb; i += blockDim.x) dst[i] = tab.b[i];
}

// pref[0][k][*]: units of the trsm of panel k (T_b - k - 1 per block);
// pref[1][k][*]: units of the herk of panel k ((T_b - k - 1)(T_b - k) / 2 per block).
__global__ void chol_prefix_kernel(const CBlk* __restrict__ tab, int nb, int Tmax, long long* __restrict__ pref) {
    const int k = blockIdx.x;
    if (threadIdx.x != 0 || k >= Tmax) return;
    long long* pt = pref + (long long)k * (nb + 1);
    long long* ph = pref + (long long)(Tmax + k) * (nb + 1);
    long long at = 0, ah = 0;
    pt[0] = 0;
    ph[0] = 0;
    for (int b = 0; b < nb; ++b) {
        const long long m = tab[b].T > k ? (long long)(tab[b].T - k - 1) : 0;
        at += m;
        ah += m * (m + 1) / 2;
        pt[b + 1] = at;
        ph[b + 1] = ah;
    }
}

// FP32 tiled copy of S~_b = S_b + lambda I (padding rows and columns hold the identity) and
// each tile's share of ||S_b||_F^2 (strictly lower entries count twice).
__global__ void __launch_bounds__(CP) chol_pack_kernel(CBufs B, const c128* __restrict__ S, int nb, double shift,
                                                       DevStatus* status) {
    __shared__ long long toffs[MAXB + 1];
    __shared__ double shd[32];
    __shared__ long long total;
    for (int b = threadIdx.x; b < nb; b += CP) toffs[b] = B.tab[b].toff;
    if (threadIdx.x == 0) {
        const CBlk& last = B.tab[nb - 1];
        total = last.toff + (long long)last.T * (last.T + 1) / 2;
        toffs[nb] = total;
    }
    __syncthreads();
    for (long long u = blockIdx.x; u < total; u += gridDim.x) {
        const int bi = find_block(toffs, nb, u);
        const CBlk blk = B.tab[bi];
        int ti, tj;
        tri_ij(u - blk.toff, &ti, &tj);
        c64* dst = B.L + u * CTE;
        double fr = 0.0;
        bool bad = false;
        for (int e = threadIdx.x; e < CTE; e += CP) {
            const int r = e / CT, c = e % CT;
            const long long R = (long long)ti * CT + r, Cc = (long long)tj * CT + c;
            c64 v;
            if (R < blk.n && Cc < blk.n) {
                if (ti > tj || c <= r) {
                    c128 s = S[blk.soff + R * blk.n + Cc];
                    if (!finite_cx(s)) bad = true;
                    const double wgt = (ti > tj || c < r) ? 2.0 : 1.0;
                    fr += wgt * cabs2(s);
                    if (R == Cc) s = mk<double>(s.re + shift, 0.0);
                    v = ccast<float>(s);
                } else {
                    v = mk<float>(0.f, 0.f);
                }
            } else {
                v = mk<float>(R == Cc ? 1.f : 0.f, 0.f);
            }
            dst[e] = v;
        }
        fr = block_sum(fr, shd);
        if (threadIdx.x == 0) B.fro[u] = fr;
        if (__syncthreads_or(bad) && threadIdx.x == 0) {
            set_status(status, NQS_ERR_NONFINITE, W_SOLVE, blk.orig);
            atomicOr(&B.flags[bi], CF_NONFINITE);
        }
    }
}

// One CTA per block: the keep-all certificate from ||S_b||_F. In capture mode a failed
// certificate is reported as NQS_ERR_RETRY by chol_out_kernel.
__global__ void __launch_bounds__(CP) chol_cert_kernel(CBufs B, int nb, double shift, double cutoff, int mode) {
    __shared__ double shd[32];
    const CBlk blk = B.tab[blockIdx.x];
    const long long nt = (long long)blk.T * (blk.T + 1) / 2;
    double s = 0.0;
    for (long long t = threadIdx.x; t < nt; t += CP) s += B.fro[blk.toff + t];
    s = block_sum(s, shd);
    if (threadIdx.x != 0) return;
    const double fro = sqrt(s) * (1.0 + 1e-12);         // >= sigma_max(S_b)
    const double upper = fro + shift;                    // >= sigma_max(S~_b)
    const double thr = mode == 0 ? cutoff * upper : cutoff;
    const double lower = shift - PSD_MARGIN * fro;       // <= sigma_min(S~_b) for a Gram S_b
    const bool ok = isfinite(fro) && lower > thr && lower > 0.0;
    if (!ok) atomicOr(&B.flags[blockIdx.x], CF_CERT);
}

// ------------------------------------------------------------------ factorization
// Diagonal tile of panel k: A = L L^H in place (unblocked, shared memory), then the
// inverse of L by columns. A non-positive or non-finite pivot flags the block (the pivot is
// replaced by 1 so that the rest stays finite).
__global__ void __launch_bounds__(CP) chol_potrf_kernel(CBufs B, int k) {
    extern __shared__ __align__(16) unsigned char smraw[];
    c64* A = reinterpret_cast<c64*>(smraw);          // [CT][LDT]
    c64* X = A + CT * LDT;                            // [CT][LDT] inverse
    __shared__ float sdinv;
    __shared__ int spiv;
    const CBlk blk = B.tab[blockIdx.x];
    if (blk.T <= k) return;
    c64* tile = B.L + tile_at(blk, k, k) * CTE;
    const int t = threadIdx.x;
    for (int e = t; e < CTE; e += CP) A[(e / CT) * LDT + (e % CT)] = tile[e];
    if (t == 0) spiv = 0;
    __syncthreads();
    const int row = t >> 2, q = t & 3;
    for (int j = 0; j < CT; ++j) {
        if (t == 0) {
            float d = A[j * LDT + j].re;
            if (!(d > 0.f) || !isfinite(d)) {
                spiv = 1;
                d = 1.f;
            }
            const float sd = sqrtf(d);
            A[j * LDT + j] = mk<float>(sd, 0.f);
            sdinv = 1.f / sd;
        }
        __syncthreads();
        if (t > j && t < CT) A[t * LDT + j] = sdinv * A[t * LDT + j];
        __syncthreads();
        // trailing update of rows > j: A[row][c] -= A[row][j] conj(A[c][j]), j < c <= row
        if (row > j) {
            const c64 a = A[row * LDT + j];
            for (int c = j + 1 + q; c <= row; c += 4) {
                const c64 b = A[c * LDT + j];
                c64 v = A[row * LDT + c];
                v.re -= a.re * b.re + a.im * b.im;
                v.im -= a.im * b.re - a.re * b.im;
                A[row * LDT + c] = v;
            }
        }
        __syncthreads();
    }
    // inverse X = L^-1 of the lower-triangular L by right-looking substitution over the whole
    // CTA: start from X = I; at step j row j of X is final once divided by L_jj, and every row
    // r > j subtracts L_rj times it (columns <= j only)
    for (int e = t; e < CT * CT; e += CP) {
        const int r = e / CT, c = e - r * CT;
        X[r * LDT + c] = mk<float>(r == c ? 1.f : 0.f, 0.f);
    }
    __syncthreads();
    for (int j = 0; j < CT; ++j) {
        const float inv = 1.f / A[j * LDT + j].re;
        if (t <= j) {
            const c64 v = X[j * LDT + t];
            X[j * LDT + t] = mk<float>(v.re * inv, v.im * inv);
        }
        __syncthreads();
        // rows j+1 .. CT-1, columns 0 .. j: (CT - 1 - j) (j + 1) entries over the CTA
        const int w = j + 1, nr = CT - 1 - j;
        for (int e = t; e < nr * w; e += CP) {
            const int r = j + 1 + e / w, c = e % w;
            const c64 l = A[r * LDT + j], xj = X[j * LDT + c];
            c64 v = X[r * LDT + c];
            v.re -= l.re * xj.re - l.im * xj.im;
            v.im -= l.re * xj.im + l.im * xj.re;
            X[r * LDT + c] = v;
        }
        __syncthreads();
    }
    c64* dinv = B.Dinv + (blk.doff + k) * CTE;
    for (int e = t; e < CTE; e += CP) {
        const int r = e / CT, c = e % CT;
        tile[e] = c <= r ? A[r * LDT + c] : mk<float>(0.f, 0.f);
        dinv[e] = X[r * LDT + c];
    }
    if (t == 0 && spiv) atomicOr(&B.flags[blockIdx.x], CF_PIVOT);
}

// Two-lane FP32 fused multiply-add (sm_100-class): (a0 b0 + c0, a1 b1 + c1), each rounded once.
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ unsigned long long pk2f(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

// C (CT x CT) = C - A B^H (SUB) or C = A B^H, row-major tiles in global memory. Thread
// (tx, ty) = (t % 16, t / 16) owns rows ty + 16 i and columns tx + 16 j (i, j < 4): the
// rows read by a warp are two broadcasts, the columns sixteen consecutive padded rows.
template <bool SUB>
__device__ __forceinline__ void tile_mul_nh(const c64* __restrict__ Ag, const c64* __restrict__ Bg, c64* Cg, c64* As,
                                            c64* Bs) {
    const int t = threadIdx.x;
    for (int e = t; e < CTE; e += CP) {
        As[(e / CT) * LDT + (e % CT)] = Ag[e];
        Bs[(e / CT) * LDT + (e % CT)] = Bg[e];
    }
    __syncthreads();
    const int tx = t & 15, ty = t >> 4;
    // accumulators as packed (Re, Im) pairs: a conj(b) = (a.re, a.im) b.re + (a.im, -a.re) b.im,
    // two two-lane FMAs per complex multiply-add
    unsigned long long acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0ull;
#pragma unroll 4
    for (int l = 0; l < CT; ++l) {
        unsigned long long a[4], as[4], br[4], bi[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const c64 v = As[(ty + 16 * i) * LDT + l];
            a[i] = pk2f(v.re, v.im);
            as[i] = pk2f(v.im, -v.re);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const c64 v = Bs[(tx + 16 * j) * LDT + l];
            br[j] = pk2f(v.re, v.re);
            bi[j] = pk2f(v.im, v.im);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = ffma2(as[i], bi[j], ffma2(a[i], br[j], acc[i][j]));
    }
    float ar[4][4], ai[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) asm("mov.b64 {%0, %1}, %2;" : "=f"(ar[i][j]), "=f"(ai[i][j]) : "l"(acc[i][j]));
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int e = (ty + 16 * i) * CT + tx + 16 * j;
            if (SUB) {
                const c64 c = Cg[e];
                Cg[e] = mk<float>(c.re - ar[i][j], c.im - ai[i][j]);
            } else {
                Cg[e] = mk<float>(ar[i][j], ai[i][j]);
            }
        }
    __syncthreads();
}

// Panel k below the diagonal: L_ik = A_ik L_kk^-H for every block with T_b > k + 1.
__global__ void __launch_bounds__(CP, 3) chol_trsm_kernel(CBufs B, int nb, int Tmax, int k) {
    extern __shared__ __align__(16) unsigned char smraw[];
    c64* As = reinterpret_cast<c64*>(smraw);
    c64* Bs = As + CT * LDT;
    const long long* pref = B.pref + (long long)k * (nb + 1);
    const long long u = blockIdx.x;
    if (u >= pref[nb]) return;
    const int bi = find_block(pref, nb, u);
    const CBlk blk = B.tab[bi];
    const int i = k + 1 + (int)(u - pref[bi]);
    c64* tile = B.L + tile_at(blk, i, k) * CTE;
    const c64* dinv = B.Dinv + (blk.doff + k) * CTE;
    tile_mul_nh<false>(tile, dinv, tile, As, Bs);
}

// Trailing update of panel k: A_ij -= L_ik L_jk^H for k < j <= i < T_b.
__global__ void __launch_bounds__(CP, 3) chol_herk_kernel(CBufs B, int nb, int Tmax, int k) {
    extern __shared__ __align__(16) unsigned char smraw[];
    c64* As = reinterpret_cast<c64*>(smraw);
    c64* Bs = As + CT * LDT;
    const long long* pref = B.pref + (long long)(Tmax + k) * (nb + 1);
    const long long u = blockIdx.x;
    if (u >= pref[nb]) return;
    const int bi = find_block(pref, nb, u);
    const CBlk blk = B.tab[bi];
    int ii, jj;
    tri_ij(u - pref[bi], &ii, &jj);
    const int i = k + 1 + ii, j = k + 1 + jj;
    tile_mul_nh<true>(B.L + tile_at(blk, i, k) * CTE, B.L + tile_at(blk, j, k) * CTE, B.L + tile_at(blk, i, j) * CTE,
                      As, Bs);
}

// ------------------------------------------------------------------ refinement
struct RefShared {
    c128 colp[4][CT];     // column partials of a residual tile
    c128 xs[2][CT];       // x of the column tile and of the row tile
    c64 v[CT];            // wavefront vector
    c64 w4[4][CT];        // column-group partials of the wavefront
    __align__(16) c64 dk[CTE];  // the unit's diagonal-tile inverse
    double rprev[MAXB];   // ||r||^2 of the previous sweep per block (the same in every CTA)
    double fn[MAXB];      // ||F||^2 per block
    int act[MAXB];        // active blocks (table order, T descending)
    int lvl[CHOL_MAXT + 1];  // prefix over tile-row levels of the active blocks
    double shd[32];
    int nact, ok, abort_;
};

__device__ bool chol_grid_sync(unsigned* bar, DevStatus* status, int* ok_s, unsigned long long budget) {
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
            const unsigned long long t0 = gtime_ns();
            while (*gen == g) {
                __nanosleep(64);
                if (gtime_ns() - t0 > budget) {
                    ok = 0;
                    set_status(status, NQS_ERR_TIMEOUT, W_SOLVE, -2);
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

// Wait until flag >= want (thread 0 polls, bounded); false on timeout.
__device__ bool wait_flag(const unsigned* flag, unsigned want, DevStatus* status, int* ok_s,
                          unsigned long long budget) {
    if (threadIdx.x == 0) {
        int ok = 1;
        const volatile unsigned* f = flag;
        if (*f < want) {
            const unsigned long long t0 = gtime_ns();
            while (*f < want) {
                __nanosleep(32);
                if (gtime_ns() - t0 > budget) {
                    ok = 0;
                    set_status(status, NQS_ERR_TIMEOUT, W_SOLVE, -3);
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

// Every thread's writes of the part are ordered before the flag: barrier, then one
// thread's device-wide fence and the flag update.
__device__ __forceinline__ void publish_flag(unsigned* flag, unsigned v) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicMax(flag, v);
    }
}

// Whether flag >= want now (thread 0 reads once; acquire fence when set); no waiting.
__device__ bool peek_flag(const unsigned* flag, unsigned want, int* ok_s) {
    if (threadIdx.x == 0) {
        const volatile unsigned* f = flag;
        const int ok = *f >= want ? 1 : 0;
        if (ok) __threadfence();
        *ok_s = ok;
    }
    __syncthreads();
    return *ok_s != 0;
}

__device__ __forceinline__ c64 ldcg64(const c64* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return mk<float>(v.x, v.y);
}
__device__ __forceinline__ c128 ldcg128(const c128* p) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return mk<double>(v.x, v.y);
}

// Residual partials of lower tile (i, j) of a block: P[i][j] += S_ij x_j (row part) and
// P[j][i] = S_ij^H x_i (column part); on the diagonal tile both parts go to P[i][i], using
// the stored lower triangle only.
__device__ void residual_tile(const CBufs& B, const c128* __restrict__ S, const CBlk& blk, int ti, int tj,
                              RefShared& sm) {
    const int t = threadIdx.x;
    const long long v0 = blk.doff * CT;
    if (t < CT) {
        sm.xs[0][t] = ldcg128(B.x + v0 + (long long)tj * CT + t);
        sm.xs[1][t] = ldcg128(B.x + v0 + (long long)ti * CT + t);
    }
    __syncthreads();
    const int n = blk.n;
    // row part: 4 threads per row, 16 columns each
    const int r = t >> 2, q = t & 3;
    const long long R = (long long)ti * CT + r;
    double pr = 0.0, pi = 0.0;
    if (R < n) {
        const c128* srow = S + blk.soff + R * n + (long long)tj * CT;
        for (int c = q; c < CT; c += 4) {
            const long long Cc = (long long)tj * CT + c;
            if (Cc >= n || (ti == tj && c > r)) continue;
            const c128 s = srow[c], xv = sm.xs[0][c];
            pr += s.re * xv.re - s.im * xv.im;
            pi += s.re * xv.im + s.im * xv.re;
        }
    }
    pr += __shfl_xor_sync(0xffffffffu, pr, 1);
    pi += __shfl_xor_sync(0xffffffffu, pi, 1);
    pr += __shfl_xor_sync(0xffffffffu, pr, 2);
    pi += __shfl_xor_sync(0xffffffffu, pi, 2);
    // column part: thread (c, g) sums rows g*16 .. g*16+15 of column c
    const int c = t & (CT - 1), g = t >> 6;
    const long long Cc = (long long)tj * CT + c;
    double cr = 0.0, ci = 0.0;
    if (Cc < n) {
        for (int rr = g * 16; rr < g * 16 + 16; ++rr) {
            const long long R2 = (long long)ti * CT + rr;
            if (R2 >= n || (ti == tj && rr <= c)) continue;  // strictly lower on the diagonal tile
            const c128 s = S[blk.soff + R2 * n + Cc], xv = sm.xs[1][rr];
            cr += s.re * xv.re + s.im * xv.im;  // conj(s) x
            ci += s.re * xv.im - s.im * xv.re;
        }
    }
    sm.colp[g][c] = mk<double>(cr, ci);
    __syncthreads();
    const long long T = blk.T;
    if (ti == tj) {
        if (q == 0) {
            const c128 cs = sm.colp[0][r] + sm.colp[1][r] + sm.colp[2][r] + sm.colp[3][r];
            B.P[(blk.poff + ti * T + ti) * CT + r] = mk<double>(pr, pi) + cs;
        }
    } else {
        if (q == 0) B.P[(blk.poff + ti * T + tj) * CT + r] = mk<double>(pr, pi);
        if (t < CT) {
            const c128 cs = sm.colp[0][t] + sm.colp[1][t] + sm.colp[2][t] + sm.colp[3][t];
            B.P[(blk.poff + (long long)tj * T + ti) * CT + t] = cs;
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(CP, 2) chol_refine_kernel(CBufs B, const c128* __restrict__ S,
                                                             const c128* __restrict__ F, int nb, int Tmax,
                                                             double shift, int maxit, unsigned long long wait_ns,
                                                             double tol, DevStatus* status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    RefShared& sm = *reinterpret_cast<RefShared*>(smraw);
    const int t = threadIdx.x;
    // x = 0; blocks already flagged (certificate, pivot, non-finite) are skipped
    for (int bi = 0; bi < nb; ++bi) {
        const CBlk blk = B.tab[bi];
        const long long len = (long long)blk.T * CT;
        for (long long e = blockIdx.x * (long long)CP + t; e < len; e += (long long)gridDim.x * CP)
            B.x[blk.doff * CT + e] = mk<double>(0.0, 0.0);
        if (blockIdx.x == 0 && t == 0) B.done[bi] = B.flags[bi] != 0 ? 1 : 0;
        if (t == 0) {
            sm.rprev[bi] = 0.0;
            sm.fn[bi] = 0.0;
        }
    }
    if (!chol_grid_sync(B.bar, status, &sm.ok, wait_ns)) return;
    for (int it = 0; it < maxit; ++it) {
        // active blocks (identical in every CTA: done[] changes only between barriers)
        if (t == 0) {
            int na = 0;
            for (int bi = 0; bi < nb; ++bi)
                if (!__ldcg(&B.done[bi])) sm.act[na++] = bi;
            sm.nact = na;
        }
        __syncthreads();
        const int na = sm.nact;
        if (na == 0) break;
        // ---- P1: residual partials over the lower tiles of the active blocks
        {
            long long base = 0;
            for (int a = 0; a < na; ++a) {
                const CBlk blk = B.tab[sm.act[a]];
                const long long nt = (long long)blk.T * (blk.T + 1) / 2;
                for (long long u = blockIdx.x - base; u < nt; u += gridDim.x) {
                    if (u < 0) continue;
                    int ti, tj;
                    tri_ij(u, &ti, &tj);
                    residual_tile(B, S, blk, ti, tj, sm);
                }
                base = (base + nt) % gridDim.x;
            }
        }
        if (!chol_grid_sync(B.bar, status, &sm.ok, wait_ns)) return;
        // ---- P2: r = F - lambda x - sum_j P[i][j] per tile row; ||r||^2 per tile row
        {
            long long base = 0;
            for (int a = 0; a < na; ++a) {
                const CBlk blk = B.tab[sm.act[a]];
                for (long long u = blockIdx.x - base; u < blk.T; u += gridDim.x) {
                    if (u < 0) continue;
                    const int ti = (int)u;
                    double nr = 0.0;
                    if (t < CT) {
                        const long long R = (long long)ti * CT + t;
                        const long long vi = blk.doff * CT + R;
                        c128 res = mk<double>(0.0, 0.0);
                        if (R < blk.n) {
                            c128 acc = mk<double>(0.0, 0.0);
                            for (int tj = 0; tj < blk.T; ++tj)
                                acc = acc + ldcg128(B.P + (blk.poff + (long long)ti * blk.T + tj) * CT + t);
                            const c128 xv = ldcg128(B.x + vi);
                            res = F[blk.off + R] - shift * xv - acc;
                        }
                        B.r[vi] = res;
                        B.r32[vi] = ccast<float>(res);
                        nr = cabs2(res);
                    }
                    nr = block_sum(nr, sm.shd);
                    if (t == 0) B.rn[blk.doff + ti] = nr;
                }
                base = (base + blk.T) % gridDim.x;
            }
        }
        if (!chol_grid_sync(B.bar, status, &sm.ok, wait_ns)) return;
        // ---- P3: convergence per block (every CTA decides the same)
        for (int a = t >> 5; a < na; a += CP / 32) {
            const int bi = sm.act[a];
            const CBlk blk = B.tab[bi];
            double s = 0.0;
            for (int i = t & 31; i < blk.T; i += 32) s += __ldcg(&B.rn[blk.doff + i]);
            s = warp_sum(s);
            if ((t & 31) == 0) {
                if (it == 0) sm.fn[bi] = s;
                const double fn = sm.fn[bi], prev = sm.rprev[bi];
                bool fin = false;
                int fl = 0;
                if (!isfinite(s)) {
                    fin = true;
                    fl = CF_NONFINITE;
                } else if (s <= tol * tol * fn) {
                    fin = true;
                } else if (it >= 1 && s <= CHOL_FLOOR * CHOL_FLOOR * fn && s > 0.0625 * prev) {
                    fin = true;  // at the residual's rounding floor: no further sweep helps
                } else if (it >= 2 && s > prev) {
                    fin = true;  // diverging: the FP32 factor is too far from S~ for this block
                    fl = CF_CONV;
                } else if (it == maxit - 1) {
                    fin = true;
                    fl = CF_CONV;
                }
                sm.rprev[bi] = s;
                sm.act[a] = fin ? -1 - bi : bi;  // marked for this CTA; written back below
                if (blockIdx.x == 0 && fl) atomicOr(&B.flags[bi], fl);
            }
        }
        __syncthreads();
        // blocks that finished this sweep take no solve; compact the active list
        if (t == 0) {
            int m = 0;
            for (int a = 0; a < na; ++a)
                if (sm.act[a] >= 0) sm.act[m++] = sm.act[a];
                else if (blockIdx.x == 0) B.done[-1 - sm.act[a]] = 1;
            sm.nact = m;
        }
        __syncthreads();
        const int nw = sm.nact;
        if (nw == 0) break;  // every block finished (the same decision in every CTA)
        // levels: lvl[i] = number of wave units of tile rows < i (active blocks with T > i)
        int Tm = 0;
        for (int a = 0; a < nw; ++a) Tm = max(Tm, B.tab[sm.act[a]].T);
        if (t == 0) {  // act[] is in table order (T descending): the blocks with T > i are a prefix
            int acc = 0, p = nw;
            for (int i = 0; i < Tm; ++i) {
                while (p > 0 && B.tab[sm.act[p - 1]].T <= i) --p;
                sm.lvl[i] = acc;
                acc += p;
            }
            sm.lvl[Tm] = acc;
        }
        __syncthreads();
        const long long U = sm.lvl[Tm];
        const unsigned gen = (unsigned)it + 1u;
        // ---- P4: forward (units 0..U-1, tile rows ascending) then backward (U..2U-1, descending).
        // A unit applies its off-diagonal tiles in the order their right-hand parts become
        // ready (forward: j = 0 .. i-1; backward: j = T-1 .. i+1), loading each tile before it
        // waits for the part it multiplies, and skips the waits once a later part is known to
        // be ready (a part is published only after every part it depends on).
        for (long long u = blockIdx.x; u < 2 * U; u += gridDim.x) {
            const bool fwd = u < U;
            const long long v = fwd ? u : u - U;
            // level i and the block: the (v - lvl[i])-th active block with T > i
            int lo = 0, hi = Tm - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sm.lvl[mid] <= v) lo = mid; else hi = mid - 1;
            }
            const int lev = lo;
            const int bi = sm.act[(int)(v - sm.lvl[lev])];
            const CBlk blk = B.tab[bi];
            const int ti = fwd ? lev : blk.T - 1 - lev;
            const long long row0 = blk.doff;  // tile-row base of the block
            {   // the diagonal tile's inverse to shared memory (needed last)
                const float4* src = reinterpret_cast<const float4*>(B.Dinv + (blk.doff + ti) * CTE);
                float4* dst = reinterpret_cast<float4*>(sm.dk);
                for (int e = t; e < CTE / 2; e += CP) dst[e] = src[e];
            }
            if (fwd) {
                // v = r_i - sum_{j < i} L_ij y_j ; y_i = Dinv_i v
                const int r = t >> 2, q = t & 3;
                float ar = 0.f, ai = 0.f;
                int known = -1;  // flags 0..known acquired
                if (ti > 0 && peek_flag(B.fflag + row0 + ti - 1, gen, &sm.ok)) known = ti - 1;
                for (int j = 0; j < ti; ++j) {
                    const c64* Lt = B.L + tile_at(blk, ti, j) * CTE + r * CT + q;
                    c64 a[CT / 4];
#pragma unroll
                    for (int m = 0; m < CT / 4; ++m) a[m] = Lt[4 * m];
                    if (j > known) {
                        if (!wait_flag(B.fflag + row0 + j, gen, status, &sm.ok, wait_ns)) return;
                        known = j;
                    }
                    const c64* yj = B.y + (row0 + j) * CT + q;
#pragma unroll
                    for (int m = 0; m < CT / 4; ++m) {
                        const c64 yv = ldcg64(yj + 4 * m);
                        ar = fmaf(a[m].re, yv.re, fmaf(-a[m].im, yv.im, ar));
                        ai = fmaf(a[m].re, yv.im, fmaf(a[m].im, yv.re, ai));
                    }
                }
                ar += __shfl_xor_sync(0xffffffffu, ar, 1);
                ai += __shfl_xor_sync(0xffffffffu, ai, 1);
                ar += __shfl_xor_sync(0xffffffffu, ar, 2);
                ai += __shfl_xor_sync(0xffffffffu, ai, 2);
                if (q == 0) {
                    const c64 rv = ldcg64(B.r32 + (row0 + ti) * CT + r);
                    sm.v[r] = mk<float>(rv.re - ar, rv.im - ai);
                }
                __syncthreads();
                float yr = 0.f, yi = 0.f;
                for (int c = q; c < CT; c += 4) {
                    const c64 a = sm.dk[r * CT + c], vv = sm.v[c];
                    yr = fmaf(a.re, vv.re, fmaf(-a.im, vv.im, yr));
                    yi = fmaf(a.re, vv.im, fmaf(a.im, vv.re, yi));
                }
                yr += __shfl_xor_sync(0xffffffffu, yr, 1);
                yi += __shfl_xor_sync(0xffffffffu, yi, 1);
                yr += __shfl_xor_sync(0xffffffffu, yr, 2);
                yi += __shfl_xor_sync(0xffffffffu, yi, 2);
                if (q == 0) B.y[(row0 + ti) * CT + r] = mk<float>(yr, yi);
                publish_flag(B.fflag + row0 + ti, gen);
            } else {
                // w = y_i - sum_{j > i} L_ji^H z_j ; z_i = Dinv_i^H w ; x_i += z_i
                const int c = t & (CT - 1), g = t >> 6;
                float ar = 0.f, ai = 0.f;
                int known = blk.T;  // flags known .. T-1 acquired
                if (ti + 1 < blk.T && peek_flag(B.bflag + row0 + ti + 1, gen, &sm.ok)) known = ti + 1;
                for (int j = blk.T - 1; j > ti; --j) {
                    const c64* Lt = B.L + tile_at(blk, j, ti) * CTE + (g * 16) * CT + c;
                    c64 a[16];
#pragma unroll
                    for (int m = 0; m < 16; ++m) a[m] = Lt[m * CT];
                    if (j < known) {
                        if (!wait_flag(B.bflag + row0 + j, gen, status, &sm.ok, wait_ns)) return;
                        known = j;
                    }
                    const c64* zj = B.z + (row0 + j) * CT + g * 16;
#pragma unroll
                    for (int m = 0; m < 16; ++m) {
                        const c64 zv = ldcg64(zj + m);  // conj(a) z
                        ar = fmaf(a[m].re, zv.re, fmaf(a[m].im, zv.im, ar));
                        ai = fmaf(a[m].re, zv.im, fmaf(-a[m].im, zv.re, ai));
                    }
                }
                if (!wait_flag(B.fflag + row0 + ti, gen, status, &sm.ok, wait_ns)) return;
                sm.w4[g][c] = mk<float>(ar, ai);
                __syncthreads();
                if (t < CT) {
                    const c64 yv = ldcg64(B.y + (row0 + ti) * CT + t);
                    const c64 s = sm.w4[0][t] + sm.w4[1][t] + sm.w4[2][t] + sm.w4[3][t];
                    sm.v[t] = yv - s;
                }
                __syncthreads();
                float zr = 0.f, zi = 0.f;
                for (int rr = g * 16; rr < g * 16 + 16; ++rr) {
                    const c64 a = sm.dk[rr * CT + c], vv = sm.v[rr];  // conj(Dinv[rr][c]) w[rr]
                    zr = fmaf(a.re, vv.re, fmaf(a.im, vv.im, zr));
                    zi = fmaf(a.re, vv.im, fmaf(-a.im, vv.re, zi));
                }
                sm.w4[g][c] = mk<float>(zr, zi);
                __syncthreads();
                if (t < CT) {
                    const c64 zz = sm.w4[0][t] + sm.w4[1][t] + sm.w4[2][t] + sm.w4[3][t];
                    B.z[(row0 + ti) * CT + t] = zz;
                    const long long xi = (row0 + ti) * CT + t;
                    B.x[xi] = ldcg128(B.x + xi) + ccast<double>(zz);
                }
                publish_flag(B.bflag + row0 + ti, gen);
            }
            __syncthreads();
        }
        if (!chol_grid_sync(B.bar, status, &sm.ok, wait_ns)) return;
    }
}

// dtheta_b = -eta x for blocks with no flag; under capture any flag is NQS_ERR_RETRY.
__global__ void chol_out_kernel(CBufs B, int nb, double eta, c128* __restrict__ dtheta, int32_t* __restrict__ n_kept,
                                bool capture, DevStatus* status) {
    const int bi = blockIdx.x;
    const CBlk blk = B.tab[bi];
    const int fl = B.flags[bi];
    if (fl != 0) {
        if (capture && threadIdx.x == 0) set_status(status, NQS_ERR_RETRY, W_SOLVE, blk.orig);
        return;
    }
    for (int k = threadIdx.x; k < blk.n; k += blockDim.x) dtheta[blk.off + k] = (-eta) * B.x[blk.doff * CT + k];
    if (threadIdx.x == 0 && n_kept) n_kept[blk.orig] = blk.n;
}

// ------------------------------------------------------------------ host side
struct CLayout {
    size_t tab, pref, L, Dinv, fro, flags, P, x, r, r32, y, z, rn, done, fflag, bflag, bar, total;
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

void build_ctab(const int64_t* off, int nb, CTab* tab) {
    int order[MAXB];
    for (int b = 0; b < nb; ++b) order[b] = b;
    for (int x = 1; x < nb; ++x) {  // by size, descending: the blocks active at a panel form a prefix
        const int v = order[x];
        const long long nv = off[v + 1] - off[v];
        int y = x - 1;
        while (y >= 0 && (off[order[y] + 1] - off[order[y]]) < nv) {
            order[y + 1] = order[y];
            --y;
        }
        order[y + 1] = v;
    }
    long long soff_of[MAXB + 1];
    soff_of[0] = 0;
    for (int b = 0; b < nb; ++b) soff_of[b + 1] = soff_of[b] + (off[b + 1] - off[b]) * (off[b + 1] - off[b]);
    tab->nb = nb;
    tab->Tmax = 0;
    long long tiles = 0, rows = 0, parts = 0;
    for (int j = 0; j < nb; ++j) {
        const int b = order[j];
        CBlk& e = tab->b[j];
        e.n = (int)(off[b + 1] - off[b]);
        e.T = (e.n + CT - 1) / CT;
        e.off = off[b];
        e.soff = soff_of[b];
        e.orig = b;
        e.pad = 0;
        e.toff = tiles;
        e.doff = rows;
        e.poff = parts;
        tiles += (long long)e.T * (e.T + 1) / 2;
        rows += e.T;
        parts += (long long)e.T * e.T;
        tab->Tmax = e.T > tab->Tmax ? e.T : tab->Tmax;
    }
    tab->tiles = tiles;
    tab->rows = rows;
    tab->parts = parts;
}

CLayout chol_layout(const CTab& tab) {
    CLayout L{};
    size_t p = 0;
    auto take = [&](size_t bytes) { size_t at = p; p += al256(bytes > 0 ? bytes : 1); return at; };
    const size_t nb = (size_t)tab.nb, rows = (size_t)tab.rows;
    L.tab = take(sizeof(CBlk) * nb);
    L.pref = take(8ull * 2 * (size_t)tab.Tmax * (nb + 1));
    L.L = take(8ull * CTE * (size_t)tab.tiles);
    L.Dinv = take(8ull * CTE * rows);
    L.fro = take(8ull * (size_t)tab.tiles);
    L.flags = take(4ull * nb);
    L.P = take(16ull * CT * (size_t)tab.parts);
    L.x = take(16ull * CT * rows);
    L.r = take(16ull * CT * rows);
    L.r32 = take(8ull * CT * rows);
    L.y = take(8ull * CT * rows);
    L.z = take(8ull * CT * rows);
    L.rn = take(8ull * rows);
    L.done = take(4ull * nb);
    L.fflag = take(4ull * rows);
    L.bflag = take(4ull * rows);
    L.bar = take(64);
    L.total = p;
    return L;
}

}  // namespace

bool chol_applicable(const int64_t* block_off, int nb) {
    for (int b = 0; b < nb; ++b)
        if ((block_off[b + 1] - block_off[b] + CT - 1) / CT > CHOL_MAXT) return false;
    return nb >= 1 && nb <= MAXB;
}

size_t chol_workspace_bytes(const int64_t* block_off, int nb) {
    if (!chol_applicable(block_off, nb)) return 0;
    CTab* tab = new (std::nothrow) CTab;
    if (!tab) return 0;
    build_ctab(block_off, nb, tab);
    const size_t total = chol_layout(*tab).total;
    delete tab;
    return total;
}

int launch_chol_solve(const c128* S, const int64_t* block_off, int nb, const c128* F, const SolveArgs& a,
                      c128* dtheta, int32_t* n_kept, void* work, size_t work_bytes, DevStatus* status,
                      cudaStream_t st, bool* ok_out) {
    *ok_out = false;
    if (!chol_applicable(block_off, nb)) return NQS_ERR_UNSUPPORTED;
    CTab* tabp = new (std::nothrow) CTab;
    if (!tabp) return NQS_ERR_INVALID_ARG;
    CTab& tab = *tabp;
    build_ctab(block_off, nb, &tab);
    const CLayout L = chol_layout(tab);
    if (work_bytes < L.total) {
        delete tabp;
        return NQS_ERR_WORKSPACE;
    }
    char* W = static_cast<char*>(work);
    CBufs B;
    B.tab = reinterpret_cast<CBlk*>(W + L.tab);
    B.pref = reinterpret_cast<long long*>(W + L.pref);
    B.L = reinterpret_cast<c64*>(W + L.L);
    B.Dinv = reinterpret_cast<c64*>(W + L.Dinv);
    B.fro = reinterpret_cast<double*>(W + L.fro);
    B.flags = reinterpret_cast<int*>(W + L.flags);
    B.P = reinterpret_cast<c128*>(W + L.P);
    B.x = reinterpret_cast<c128*>(W + L.x);
    B.r = reinterpret_cast<c128*>(W + L.r);
    B.r32 = reinterpret_cast<c64*>(W + L.r32);
    B.y = reinterpret_cast<c64*>(W + L.y);
    B.z = reinterpret_cast<c64*>(W + L.z);
    B.rn = reinterpret_cast<double*>(W + L.rn);
    B.done = reinterpret_cast<int*>(W + L.done);
    B.fflag = reinterpret_cast<unsigned*>(W + L.fflag);
    B.bflag = reinterpret_cast<unsigned*>(W + L.bflag);
    B.bar = reinterpret_cast<unsigned*>(W + L.bar);
    const int Tmax = tab.Tmax;
    int Ts[MAXB];
    for (int j = 0; j < nb; ++j) Ts[j] = tab.b[j].T;
    const long long total_tiles = tab.tiles;
    const long long rows = tab.rows;
    delete tabp;

    auto ck = [&](void) { return cudaGetLastError() == cudaSuccess ? NQS_OK : NQS_ERR_CUDA; };
    // set-up: table, unit prefixes, flags and wave flags cleared
    {
        CTab* t2 = new (std::nothrow) CTab;
        if (!t2) return NQS_ERR_INVALID_ARG;
        build_ctab(block_off, nb, t2);
        count_launch();
        chol_upload_kernel<<<1, 256, 0, st>>>(*t2, const_cast<CBlk*>(B.tab));
        delete t2;
    }
    if (cudaMemsetAsync(B.flags, 0, 4ull * nb, st) != cudaSuccess) return NQS_ERR_CUDA;
    if (cudaMemsetAsync(B.fflag, 0, 4ull * rows, st) != cudaSuccess) return NQS_ERR_CUDA;
    if (cudaMemsetAsync(B.bflag, 0, 4ull * rows, st) != cudaSuccess) return NQS_ERR_CUDA;
    if (cudaMemsetAsync(B.bar, 0, 64, st) != cudaSuccess) return NQS_ERR_CUDA;
    count_launch();
    chol_prefix_kernel<<<Tmax, 32, 0, st>>>(B.tab, nb, Tmax, const_cast<long long*>(B.pref));
    // FP32 tiled copy of S~ and the certificate
    {
        const long long g = total_tiles < 8192 ? total_tiles : 8192;
        count_launch();
        chol_pack_kernel<<<(unsigned)g, CP, 0, st>>>(B, S, nb, a.shift, status);
        count_launch();
        chol_cert_kernel<<<nb, CP, 0, st>>>(B, nb, a.shift, a.cutoff, a.cutoff_mode);
    }
    int rc = ck();
    if (rc) return rc;
    // factorization, panel by panel
    if (a.ev_trd_start) cudaEventRecord(a.ev_trd_start, st);
    const int smem_potrf = 2 * CT * LDT * (int)sizeof(c64);
    const int smem_mul = 2 * CT * LDT * (int)sizeof(c64);
    if (cudaFuncSetAttribute(chol_potrf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_potrf) !=
            cudaSuccess ||
        cudaFuncSetAttribute(chol_trsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_mul) != cudaSuccess ||
        cudaFuncSetAttribute(chol_herk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_mul) != cudaSuccess)
        return NQS_ERR_CUDA;
    for (int k = 0; k < Tmax; ++k) {
        int nact = 0;
        long long ut = 0, uh = 0;
        for (int j = 0; j < nb; ++j)
            if (Ts[j] > k) {
                ++nact;
                const long long m = Ts[j] - k - 1;
                ut += m;
                uh += m * (m + 1) / 2;
            }
        count_launch();
        chol_potrf_kernel<<<nact, CP, smem_potrf, st>>>(B, k);
        if (ut > 0) {
            count_launch();
            chol_trsm_kernel<<<(unsigned)ut, CP, smem_mul, st>>>(B, nb, Tmax, k);
        }
        if (uh > 0) {
            count_launch();
            chol_herk_kernel<<<(unsigned)uh, CP, smem_mul, st>>>(B, nb, Tmax, k);
        }
    }
    rc = ck();
    if (rc) return rc;
    if (a.ev_trd_done) cudaEventRecord(a.ev_trd_done, st);
    // refinement: one cooperative launch
    {
        const int smem_ref = (int)sizeof(RefShared);
        if (cudaFuncSetAttribute(chol_refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_ref) !=
            cudaSuccess)
            return NQS_ERR_CUDA;
        int dev = 0, sms = 0, per = 0, coop = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, chol_refine_kernel, CP, smem_ref) != cudaSuccess ||
            per < 1)
            return NQS_ERR_CUDA;
        const int grid = sms * (per < 2 ? per : 2);
        const Limits lim = limits();
        int nbv = nb, tm = Tmax, maxit = lim.ref_maxit;
        double shift = a.shift;
        unsigned long long wait_ns = lim.wait_ns;
        double tol = a.ref_tol > 0.0 ? a.ref_tol : CHOL_TOL;
        void* args[] = {&B, (void*)&S, (void*)&F, &nbv, &tm, &shift, &maxit, &wait_ns, &tol, &status};
        count_launch();
        if (cudaLaunchCooperativeKernel((const void*)chol_refine_kernel, dim3(grid), dim3(CP), args, smem_ref, st) !=
            cudaSuccess)
            return NQS_ERR_CUDA;
    }
    count_launch();
    chol_out_kernel<<<nb, 256, 0, st>>>(B, nb, a.eta, dtheta, n_kept, a.no_host_sync, status);
    rc = ck();
    if (rc) return rc;
    if (a.no_host_sync) {
        *ok_out = true;  // a failure is reported on the device (NQS_ERR_RETRY)
        return NQS_OK;
    }
    int fl[MAXB];
    if (cudaMemcpyAsync(fl, B.flags, sizeof(int) * nb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return NQS_ERR_CUDA;
    bool ok = true;
    for (int j = 0; j < nb; ++j) ok = ok && fl[j] == 0;
    *ok_out = ok;
    return NQS_OK;
}

}  // namespace nqs
