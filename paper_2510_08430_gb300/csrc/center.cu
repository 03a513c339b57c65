// Means, centring and force (second form of Eq. 2; Sec. 2 force):
//   <E> = sum_s w_s E_loc(s),  e_s = E_loc(s) - <E>,
//   <O_k> = sum_s w_s O_k(s),  dO_k(s) = O_k(s) - <O_k>,
//   F_k = sum_s w_s conj(dO_k(s)) e_s.
// One CTA per parameter row (a contiguous run of samples): pass 1 reduces the
// mean, pass 2 re-reads the row (from L2) to write dO and reduce F. All sums
// accumulate in FP64. In split mode pass 2 writes BF16 hi/lo planes of dO
// (rows 2k = Re, 2k+1 = Im; sqrt(w_s) folded in when weights are given) for
// the tensor-core Gram instead of writing dO back.
#include <cuda_bf16.h>
#include "internal.cuh"

namespace nqs {

// Inputs of one shard of a sample-sharded step: the global means (instead of the shard's
// own) and the weight of every sample (1/N over all shards). Both unused when NULL/0.
struct ShardArgs {
    const c128* mean_in;
    double wconst;
};

// e = E_loc - <E> with the global <E> of a sample-sharded step.
__global__ void ecenter_kernel(const c128* __restrict__ eloc, long long ns, const c128* __restrict__ emean,
                               c128* __restrict__ e) {
    const c128 m = emean[0];
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < ns; s += (long long)gridDim.x * blockDim.x)
        e[s] = eloc[s] - m;
}

// out[p] = sum_s X[p][s] (FP64), the per-shard sums behind the global means.
template <typename R>
__global__ void __launch_bounds__(256) rowsum_kernel(const cx<R>* __restrict__ X, long long ldx, long long ns,
                                                      c128* __restrict__ out) {
    __shared__ double sh[32];
    const cx<R>* row = X + blockIdx.x * ldx;
    double re = 0.0, im = 0.0;
    for (long long s = threadIdx.x; s < ns; s += blockDim.x) {
        re += (double)row[s].re;
        im += (double)row[s].im;
    }
    re = block_sum(re, sh);
    im = block_sum(im, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = mk<double>(re, im);
}

cudaError_t launch_shard_sums(int prec, const void* O, long long ldo, long long ns, long long np, const c128* eloc,
                              c128* osum, c128* esum, cudaStream_t st) {
    count_launch();
    if (prec == NQS_FP32)
        rowsum_kernel<float><<<(unsigned)np, 256, 0, st>>>((const c64*)O, ldo, ns, osum);
    else
        rowsum_kernel<double><<<(unsigned)np, 256, 0, st>>>((const c128*)O, ldo, ns, osum);
    count_launch();
    rowsum_kernel<double><<<1, 256, 0, st>>>(eloc, ns, ns, esum);
    return cudaGetLastError();
}

// Global means of a sample-sharded step from the all-reduced shard sums:
// means[k] = osum[k] / n_total (k < n_p), means[n_p] = esum[0] / n_total.
__global__ void sums_to_means_kernel(const c128* __restrict__ osum, const c128* __restrict__ esum, long long np,
                                     double inv_n, c128* __restrict__ means) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k <= np; k += (long long)gridDim.x * blockDim.x)
        means[k] = inv_n * (k < np ? osum[k] : esum[0]);
}

cudaError_t launch_sums_to_means(const c128* osum, const c128* esum, long long np, long long n_total, c128* means,
                                 cudaStream_t st) {
    count_launch();
    const long long g = (np + 256) / 256;
    sums_to_means_kernel<<<(unsigned)(g < 1024 ? g : 1024), 256, 0, st>>>(osum, esum, np, 1.0 / (double)n_total,
                                                                           means);
    return cudaGetLastError();
}

cudaError_t launch_ecenter(const c128* eloc, long long ns, const c128* emean, c128* e, cudaStream_t st) {
    count_launch();
    ecenter_kernel<<<(unsigned)((ns + 255) / 256 < 1024 ? (ns + 255) / 256 : 1024), 256, 0, st>>>(eloc, ns, emean, e);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(1024) emean_kernel(const c128* __restrict__ eloc, const double* __restrict__ w,
                                                      long long ns, c128* __restrict__ emean,
                                                      c128* __restrict__ e, DevStatus* status) {
    __shared__ double sh[32];
    __shared__ double res[2];
    double re = 0.0, im = 0.0;
    const double u = 1.0 / (double)ns;
    for (long long s = threadIdx.x; s < ns; s += blockDim.x) {
        const double ws = w ? w[s] : u;
        re = fma(ws, eloc[s].re, re);
        im = fma(ws, eloc[s].im, im);
    }
    re = block_sum(re, sh);
    im = block_sum(im, sh);
    if (threadIdx.x == 0) {
        res[0] = re;
        res[1] = im;
        if (emean) emean[0] = mk<double>(re, im);
        if (!isfinite(re) || !isfinite(im)) set_status(status, NQS_ERR_NONFINITE, W_CENTER, -1);
    }
    __syncthreads();
    const c128 m = mk<double>(res[0], res[1]);
    for (long long s = threadIdx.x; s < ns; s += blockDim.x) e[s] = eloc[s] - m;
}

// Element-wise split x ~ x1 + x2 (+ x3): each term the BF16 rounding of the remainder.
template <int NS>
__device__ __forceinline__ void bf16_split(double x, __nv_bfloat16 (&p)[3]) {
    double r = x;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        p[i] = __double2bfloat16(r);
        r -= (double)__bfloat162float(p[i]);
    }
}

template <typename R>
__global__ void __launch_bounds__(256) center_kernel(cx<R>* __restrict__ O, long long ldo, long long ns,
                                                      const double* __restrict__ w, const c128* __restrict__ e,
                                                      c128* __restrict__ F, c128* __restrict__ Omean,
                                                      ShardArgs sa, DevStatus* status) {
    __shared__ double sh[32];
    const long long p = blockIdx.x;
    cx<R>* row = O + p * ldo;
    const double u = 1.0 / (double)ns;
    const double uw = sa.wconst > 0.0 ? sa.wconst : u;  // weight of every sample when w is NULL
    double mr = 0.0, mi = 0.0;
    for (long long s = threadIdx.x; s < (sa.mean_in ? 0 : ns); s += blockDim.x) {
        const cx<R> v = row[s];
        const double ws = w ? w[s] : 1.0;
        mr = fma(ws, (double)v.re, mr);
        mi = fma(ws, (double)v.im, mi);
    }
    mr = block_sum(mr, sh);
    mi = block_sum(mi, sh);
    if (!w) {
        mr *= u;
        mi *= u;
    }
    if (sa.mean_in) {  // global mean of a sample-sharded step
        mr = sa.mean_in[p].re;
        mi = sa.mean_in[p].im;
    }
    double fr = 0.0, fi = 0.0;
    for (long long s = threadIdx.x; s < ns; s += blockDim.x) {
        const cx<R> v = row[s];
        const double ws = w ? w[s] : uw;
        const cx<R> d = mk<R>((R)((double)v.re - mr), (R)((double)v.im - mi));
        row[s] = d;
        const c128 es = e[s];
        fr = fma(ws, fma((double)d.re, es.re, (double)d.im * es.im), fr);
        fi = fma(ws, fma((double)d.re, es.im, -(double)d.im * es.re), fi);
    }
    fr = block_sum(fr, sh);
    fi = block_sum(fi, sh);
    if (threadIdx.x == 0) {
        F[p] = mk<double>(fr, fi);
        if (Omean) Omean[p] = mk<double>(mr, mi);
        if (!(isfinite(mr) && isfinite(mi) && isfinite(fr) && isfinite(fi)))
            set_status(status, NQS_ERR_NONFINITE, W_CENTER, p);
    }
}

// Split mode (O is c128, left unchanged): mean and force in FP64, then NS BF16 split
// planes of sqrt(w) dO (rows 2k = Re, 2k+1 = Im; zero beyond n_s up to ldk).
template <int NS>
__global__ void __launch_bounds__(256) center_split_kernel(const c128* __restrict__ O, long long ldo, long long ns,
                                                            const double* __restrict__ w,
                                                            const c128* __restrict__ e, c128* __restrict__ F,
                                                            c128* __restrict__ Omean, __nv_bfloat16* __restrict__ pl0,
                                                            __nv_bfloat16* __restrict__ pl1,
                                                            __nv_bfloat16* __restrict__ pl2, long long ldk,
                                                            double* __restrict__ diag, ShardArgs sa,
                                                            DevStatus* status) {
    __shared__ double sh[32];
    const long long p = blockIdx.x;
    const c128* row = O + p * ldo;
    const double u = 1.0 / (double)ns;
    const double uw = sa.wconst > 0.0 ? sa.wconst : u;  // weight of every sample when w is NULL
    double mr = 0.0, mi = 0.0;
    for (long long s = threadIdx.x; s < (sa.mean_in ? 0 : ns); s += blockDim.x) {
        const c128 v = row[s];
        const double ws = w ? w[s] : 1.0;
        mr = fma(ws, v.re, mr);
        mi = fma(ws, v.im, mi);
    }
    mr = block_sum(mr, sh);
    mi = block_sum(mi, sh);
    if (!w) {
        mr *= u;
        mi *= u;
    }
    if (sa.mean_in) {  // global mean of a sample-sharded step
        mr = sa.mean_in[p].re;
        mi = sa.mean_in[p].im;
    }
    double fr = 0.0, fi = 0.0, dg = 0.0;
    __nv_bfloat16* pls[3] = {pl0, pl1, pl2};
    for (long long s = threadIdx.x; s < ldk; s += blockDim.x) {
        double dr = 0.0, di = 0.0;
        if (s < ns) {
            const c128 v = row[s];
            const double ws = w ? w[s] : uw;
            dr = v.re - mr;
            di = v.im - mi;
            const c128 es = e[s];
            fr = fma(ws, fma(dr, es.re, di * es.im), fr);
            fi = fma(ws, fma(dr, es.im, -di * es.re), fi);
            dg = fma(ws, fma(dr, dr, di * di), dg);
            if (w) {
                const double sw = sqrt(ws);
                dr *= sw;
                di *= sw;
            }
        }
        __nv_bfloat16 qr[3], qi[3];
        bf16_split<NS>(dr, qr);
        bf16_split<NS>(di, qi);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            pls[q][(2 * p) * ldk + s] = qr[q];
            pls[q][(2 * p + 1) * ldk + s] = qi[q];
        }
    }
    fr = block_sum(fr, sh);
    fi = block_sum(fi, sh);
    dg = block_sum(dg, sh);
    if (threadIdx.x == 0) {
        F[p] = mk<double>(fr, fi);
        if (Omean) Omean[p] = mk<double>(mr, mi);
        diag[p] = dg;
        if (!(isfinite(mr) && isfinite(mi) && isfinite(fr) && isfinite(fi)))
            set_status(status, NQS_ERR_NONFINITE, W_CENTER, p);
    }
}

// S_b[k][k] = sum_s w_s |dO_k(s)|^2 computed in FP64 by the split centring kernel.
__global__ void set_diag_kernel(c128* __restrict__ S, const GramTable tab, const double* __restrict__ diag) {
    const int b = blockIdx.y;
    const GBlk blk = tab.b[b];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < blk.n; k += gridDim.x * blockDim.x)
        S[blk.s_off + (long long)k * blk.n + k] = mk<double>(diag[blk.row0 + k], 0.0);
}

cudaError_t launch_set_diag(c128* S, const GramTable& tab, const double* diag, cudaStream_t st) {
    count_launch();
    set_diag_kernel<<<dim3(32, tab.nb), 256, 0, st>>>(S, tab, diag);
    return cudaGetLastError();
}

cudaError_t launch_emean(const c128* eloc, const double* w, long long ns, c128* emean, c128* e,
                         DevStatus* status, cudaStream_t st) {
    count_launch();
    emean_kernel<<<1, 1024, 0, st>>>(eloc, w, ns, emean, e, status);
    return cudaGetLastError();
}

// Grouped error-free split (O is c128, unchanged): for every parameter row and every
// group of GROUP = 32 samples, E = exponent of the group's max |Re|, |Im| of sqrt(w) dO;
// each value t = x 2^-E (|t| < 1) is rounded once to N = rint(t 2^39) and N is written in
// balanced base 256, N = sum_q d_q 2^(8(4-q)) with |d_q| <= 128; slice q is the BF16
// value d_q 2^-(8q+7) (an integer of at most 8 bits times a power of two, exact in
// BF16). Products of slices of one group then lie on a common grid: a sum of 32 leading
// products is below 2^19 grid units and exact in FP32, so the tensor-core Gram accumulates
// a whole group in tensor memory before its epilogue scales it by 2^(E_k + E_l).

// Balanced base-256 digits of |N| < 2^39, most significant first.
__device__ __forceinline__ void digits5(long long N, int (&d)[5]) {
#pragma unroll
    for (int q = 4; q >= 1; --q) {
        const int lo = (int)(((N + 128) & 255) - 128);
        d[q] = lo;
        N = (N - lo) >> 8;
    }
    d[0] = (int)N;
}
// round(x 2^k) to the nearest integer, ties to even, from the bits of x with integer
// operations only (GB300's FP64 rate is a small fraction of its integer rate); exact for
// |x 2^k| < 2^62. Equals __double2ll_rn(x * 2^k) wherever x * 2^k is exact.
__device__ __forceinline__ long long scaled_round(double x, int k) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return 0;  // zero or subnormal: far below one unit for every k used here
    const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);  // x = m 2^(e - 1075)
    const int sh = 1075 - e - k;                                 // x 2^k = m 2^-sh
    long long q;
    if (sh <= 0) {
        q = m << (-sh);
    } else if (sh > 54) {
        q = 0;
    } else {
        const long long rem = m & ((1LL << sh) - 1), half = 1LL << (sh - 1);
        q = m >> sh;
        q += (rem > half || (rem == half && (q & 1))) ? 1 : 0;
    }
    return b < 0 ? -q : q;
}
// |x| as an integer: for non-negative doubles the bit patterns order like the values
__device__ __forceinline__ long long abs_bits(double x) { return __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL; }

constexpr int GROUP = GRAM_GROUP;  // samples per exponent group: one warp, one sample per lane
static_assert(GROUP == 32, "one warp per exponent group");
// The five slices (integers of at most 8 bits scaled by 2^-7, 2^-15, ..., 2^-39) of column c
// of real rows r (Re) and r + 1 (Im) into the three plane units: slices 1-2 and 3-4 in rows
// of 2 ldk (column 64 (c / 32) + 32 h + c % 32 for the pair's slice h), slice 5 in rows of ldk.
__device__ __forceinline__ void store_slices(__nv_bfloat16* __restrict__ p12, __nv_bfloat16* __restrict__ p34,
                                             __nv_bfloat16* __restrict__ p5, long long r, long long c, long long ldk,
                                             const int (&dr5)[5], const int (&di5)[5]) {
    const float qs[5] = {0x1p-7f, 0x1p-15f, 0x1p-23f, 0x1p-31f, 0x1p-39f};
    const long long cp = 64 * (c / GROUP) + (c % GROUP);
    __nv_bfloat16* u[2] = {p12, p34};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        __nv_bfloat16* b = u[q >> 1] + 32 * (q & 1) + cp;
        b[r * 2 * ldk] = __float2bfloat16_rn((float)dr5[q] * qs[q]);
        b[(r + 1) * 2 * ldk] = __float2bfloat16_rn((float)di5[q] * qs[q]);
    }
    p5[r * ldk + c] = __float2bfloat16_rn((float)dr5[4] * qs[4]);
    p5[(r + 1) * ldk + c] = __float2bfloat16_rn((float)di5[4] * qs[4]);
}

__global__ void __launch_bounds__(256) center_group_kernel(const c128* __restrict__ O, long long ldo, long long ns,
                                                            const double* __restrict__ w,
                                                            const c128* __restrict__ e, c128* __restrict__ F,
                                                            c128* __restrict__ Omean, __nv_bfloat16* __restrict__ p12,
                                                            __nv_bfloat16* __restrict__ p34,
                                                            __nv_bfloat16* __restrict__ p5, int8_t* __restrict__ gexp,
                                                            long long gstride, long long ldk, double* __restrict__ diag,
                                                            ShardArgs sa, DevStatus* status) {
    __shared__ double sh[32];
    const long long p = blockIdx.x;
    const c128* row = O + p * ldo;
    const double u = 1.0 / (double)ns;
    const double uw = sa.wconst > 0.0 ? sa.wconst : u;  // weight of every sample when w is NULL
    double mr = 0.0, mi = 0.0;
#pragma unroll 4
    for (long long s = threadIdx.x; s < (sa.mean_in ? 0 : ns); s += blockDim.x) {
        const c128 v = row[s];
        const double ws = w ? w[s] : 1.0;
        mr = fma(ws, v.re, mr);
        mi = fma(ws, v.im, mi);
    }
    mr = block_sum(mr, sh);
    mi = block_sum(mi, sh);
    if (!w) {
        mr *= u;
        mi *= u;
    }
    if (sa.mean_in) {  // global mean of a sample-sharded step
        mr = sa.mean_in[p].re;
        mi = sa.mean_in[p].im;
    }
    // with uniform weights the sums run unweighted and are scaled once at the end (fewer
    // FP64 operations per element)
    double fr = 0.0, fi = 0.0, dg = 0.0;
    const int lane = threadIdx.x & 31;
    // blockDim.x is a multiple of 32 and ldk of GROUP: the samples of a group are one warp
    // (the trip count is warp-uniform)
    for (long long s = threadIdx.x; s < ldk; s += blockDim.x) {
        double dr = 0.0, di = 0.0;
        if (s < ns) {
            const c128 v = row[s];
            dr = v.re - mr;
            di = v.im - mi;
            const c128 es = e[s];
            if (w) {
                const double ws = w[s];
                fr = fma(ws, fma(dr, es.re, di * es.im), fr);
                fi = fma(ws, fma(dr, es.im, -di * es.re), fi);
                dg = fma(ws, fma(dr, dr, di * di), dg);
                const double sw = sqrt(ws);
                dr *= sw;
                di *= sw;
            } else {
                fr = fma(dr, es.re, fma(di, es.im, fr));
                fi = fma(dr, es.im, fma(-di, es.re, fi));
                dg = fma(dr, dr, fma(di, di, dg));
            }
        }
        long long mx = abs_bits(dr) > abs_bits(di) ? abs_bits(dr) : abs_bits(di);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long y = __shfl_xor_sync(0xffffffffu, mx, o);
            mx = y > mx ? y : mx;
        }
        // E with mx = m 2^E, m in [0.5, 1) (frexp convention), from the exponent bits
        int ex = (int)((mx >> 52) & 0x7ff) - 1022;
        ex = mx != 0 ? ex : 0;
        ex = ex < -120 ? -120 : (ex > 120 ? 120 : ex);
        if (lane == 0) gexp[(s / GROUP) * gstride + p] = (int8_t)ex;
        int dr5[5], di5[5];
        digits5(scaled_round(dr, 39 - ex), dr5);  // round(dr 2^(39 - E))
        digits5(scaled_round(di, 39 - ex), di5);
        store_slices(p12, p34, p5, 2 * p, s, ldk, dr5, di5);
    }
    fr = block_sum(fr, sh);
    fi = block_sum(fi, sh);
    dg = block_sum(dg, sh);
    if (!w) {
        fr *= uw;
        fi *= uw;
        dg *= uw;
    }
    if (threadIdx.x == 0) {
        F[p] = mk<double>(fr, fi);
        if (Omean) Omean[p] = mk<double>(mr, mi);
        diag[p] = dg;
        if (!(isfinite(mr) && isfinite(mi) && isfinite(fr) && isfinite(fi)))
            set_status(status, NQS_ERR_NONFINITE, W_CENTER, p);
    }
}

// Sample-major grouped error-free split of a centred block (sample-space Gram of a block
// wider than the sample count): for dO (c128, parameter-major [n_b][ldo], already centred)
// the planes hold rows 2s = Re dO(s), 2s+1 = Im dO(s) along the block's parameters k
// (ldk >= n_b, zero beyond n_b), split into five BF16 slices exactly as center_group_kernel
// does along samples, with one exponent per (sample, group of GROUP parameters):
// gexp[k / GROUP][s]. diag[s] += sum_k |dO_k(s)|^2 / ns (FP64; diag zeroed by the caller).
// One CTA per 32 x 32 (parameter, sample) tile; warp w takes samples w, w + 8, w + 16, w + 24
// of the tile, lane r its parameter k0 + r.
__global__ void __launch_bounds__(256) transpose_group_kernel(const c128* __restrict__ dO, long long ldo, long long ns,
                                                               long long nb, __nv_bfloat16* __restrict__ p12,
                                                               __nv_bfloat16* __restrict__ p34,
                                                               __nv_bfloat16* __restrict__ p5,
                                                               int8_t* __restrict__ gexp, long long ldk,
                                                               double* __restrict__ diag) {
    __shared__ c128 t[32][33];
    const long long s0 = (long long)blockIdx.x * 32, k0 = (long long)blockIdx.y * 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int r = wid; r < 32; r += 8) {
        const long long k = k0 + r, s = s0 + lane;
        t[r][lane] = (k < nb && s < ns) ? dO[k * ldo + s] : mk<double>(0.0, 0.0);
    }
    __syncthreads();
    const double inv_ns = 1.0 / (double)ns;
    for (int c = wid; c < 32; c += 8) {
        const long long s = s0 + c;
        if (s >= ns) continue;  // warp-uniform
        const c128 v = t[lane][c];
        const double dr = v.re, di = v.im;
        double mx = fmax(fabs(dr), fabs(di));
        double d2 = dr * dr + di * di;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        }
        int ex = (int)((__double_as_longlong(mx) >> 52) & 0x7ff) - 1022;
        ex = mx > 0.0 ? ex : 0;
        ex = ex < -120 ? -120 : (ex > 120 ? 120 : ex);
        if (lane == 0) {
            gexp[(k0 / GROUP) * ns + s] = (int8_t)ex;
            if (d2 != 0.0) atomicAdd(diag + s, d2 * inv_ns);
        }
        int dr5[5], di5[5];
        digits5(scaled_round(dr, 39 - ex), dr5);  // round(dr 2^(39 - E))
        digits5(scaled_round(di, 39 - ex), di5);
        const long long k = k0 + lane;
        if (k < ldk) store_slices(p12, p34, p5, 2 * s, k, ldk, dr5, di5);
    }
}

cudaError_t launch_transpose_group(const c128* dO, long long ldo, long long ns, long long nb, void* const* planes,
                                   int8_t* gexp, long long ldk, double* diag, cudaStream_t st) {
    if (ldk % 64 != 0 || ldk < nb) return cudaErrorInvalidValue;
    if (cudaMemsetAsync(diag, 0, sizeof(double) * ns, st) != cudaSuccess) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((ns + 31) / 32), (unsigned)(ldk / 32));
    count_launch();
    transpose_group_kernel<<<grid, 256, 0, st>>>(dO, ldo, ns, nb, (__nv_bfloat16*)planes[0], (__nv_bfloat16*)planes[1],
                                                 (__nv_bfloat16*)planes[2], gexp, ldk, diag);
    return cudaGetLastError();
}

// out[k] = sum_s conj(O[k][s]) g[s] (vector-Jacobian product of ln psi, FP64 accumulation).
template <typename R>
__global__ void __launch_bounds__(256) vjp_kernel(const cx<R>* __restrict__ O, long long ldo, long long ns,
                                                   const c128* __restrict__ g, c128* __restrict__ out) {
    __shared__ double sh[32];
    const long long p = blockIdx.x;
    const cx<R>* row = O + p * ldo;
    c128 acc = mk<double>(0.0, 0.0);
    for (long long s = threadIdx.x; s < ns; s += blockDim.x) cmacc(acc, ccast<double>(row[s]), g[s]);
    acc.re = block_sum(acc.re, sh);
    acc.im = block_sum(acc.im, sh);
    if (threadIdx.x == 0) out[p] = acc;
}

cudaError_t launch_vjp(int prec, const void* O, long long ldo, long long ns, long long np, const c128* g, c128* out,
                       cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    count_launch();
    if (prec == NQS_FP32)
        vjp_kernel<float><<<(unsigned)np, 256, 0, st>>>((const c64*)O, ldo, ns, g, out);
    else
        vjp_kernel<double><<<(unsigned)np, 256, 0, st>>>((const c128*)O, ldo, ns, g, out);
    return cudaGetLastError();
}

cudaError_t launch_center(int prec, int nsplit, void* O, long long ldo, long long ns, long long np,
                          const double* w, const c128* e, c128* F, c128* Omean, void* const* planes, long long ldk,
                          double* diag, int8_t* gexp, long long gstride, DevStatus* status, cudaStream_t st,
                          const c128* mean_in, double wconst) {
    const ShardArgs sa{mean_in, wconst};
    if (np <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)np;
    if (nsplit == 5) {
        count_launch();
        center_group_kernel<<<grid, 256, 0, st>>>((const c128*)O, ldo, ns, w, e, F, Omean,
                                                  (__nv_bfloat16*)planes[0], (__nv_bfloat16*)planes[1],
                                                  (__nv_bfloat16*)planes[2], gexp, gstride, ldk, diag, sa, status);
    } else if (nsplit == 2 || nsplit == 3) {
        __nv_bfloat16* p0 = (__nv_bfloat16*)planes[0];
        __nv_bfloat16* p1 = (__nv_bfloat16*)planes[1];
        __nv_bfloat16* p2 = nsplit == 3 ? (__nv_bfloat16*)planes[2] : nullptr;
        count_launch();
        if (nsplit == 2)
            center_split_kernel<2><<<grid, 256, 0, st>>>((const c128*)O, ldo, ns, w, e, F, Omean, p0, p1, p2, ldk,
                                                         diag, sa, status);
        else
            center_split_kernel<3><<<grid, 256, 0, st>>>((const c128*)O, ldo, ns, w, e, F, Omean, p0, p1, p2, ldk,
                                                         diag, sa, status);
    } else if (prec == NQS_FP64) {
        count_launch();
        center_kernel<double><<<grid, 256, 0, st>>>((c128*)O, ldo, ns, w, e, F, Omean, sa, status);
    } else {
        count_launch();
        center_kernel<float><<<grid, 256, 0, st>>>((c64*)O, ldo, ns, w, e, F, Omean, sa, status);
    }
    return cudaGetLastError();
}

}  // namespace nqs
