// Local energies (Eq. 1) of the bond Hamiltonians of Sec. 3:
//   E_loc(x) = c sum_b J_b [ x_i x_j + [x_i != x_j] 2 sign psi(x^{ij}) / psi(x) ].
// Integer stage: per sample, the anti-aligned bonds in bond order (warp ballots
// over a shared-memory bond table) -> counts, exclusive scan, connection list.
// Float stage: every connected configuration is pushed through the network in
// tiles of TR rows with activations in shared memory; the first layer is
// updated incrementally from the stored pre-activation of the parent sample,
// z' = z - 2 x_i W[:, i] - 2 x_j W[:, j].
#include "internal.cuh"

namespace nqs {

constexpr int CONN_WARPS = 8;

// Bond (i, j) as read from the caller's table; a bond with i == j or an index outside
// [0, N) becomes (-1, -1), which no stage treats as anti-aligned or reads spins for.
__device__ __forceinline__ int2 checked_bond(const int32_t* __restrict__ bij, int b, int N, bool* bad) {
    const int i = bij[2 * b], j = bij[2 * b + 1];
    if (i < 0 || i >= N || j < 0 || j >= N || i == j) {
        *bad = true;
        return make_int2(-1, -1);
    }
    return make_int2(i, j);
}
__device__ __forceinline__ bool anti_aligned(const int8_t* row, int2 bd) {
    return bd.x >= 0 && row[bd.x] != row[bd.y];
}

// Counts the anti-aligned bonds of every sample; also validates the bond table and
// records NQS_ERR_INVALID_ARG (detail: first bad bond index seen) for a bad bond.
__global__ void __launch_bounds__(256) conn_count_kernel(const int8_t* __restrict__ x, long long ns,
                                                          int N, int nb, const int32_t* __restrict__ bij,
                                                          int32_t* __restrict__ cnt, DevStatus* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int2* bonds = reinterpret_cast<int2*>(smem_raw);
    int8_t* rowbuf = reinterpret_cast<int8_t*>(bonds + nb);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        bool bad = false;
        bonds[b] = checked_bond(bij, b, N, &bad);
        if (bad && blockIdx.x == 0) set_status(status, NQS_ERR_INVALID_ARG, W_ELOC, b);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int8_t* row = rowbuf + wid * N;
    for (long long s = (long long)blockIdx.x * CONN_WARPS + wid; s < ns; s += (long long)gridDim.x * CONN_WARPS) {
        for (int k = lane; k < N; k += 32) row[k] = x[s * N + k];
        __syncwarp();
        int total = 0;
        for (int b0 = 0; b0 < nb; b0 += 32) {
            const int b = b0 + lane;
            bool anti = false;
            if (b < nb) anti = anti_aligned(row, bonds[b]);
            total += __popc(__ballot_sync(0xffffffffu, anti));
        }
        if (lane == 0) cnt[s] = total;
        __syncwarp();
    }
}

__global__ void __launch_bounds__(256) conn_fill_kernel(const int8_t* __restrict__ x, long long ns, int N,
                                                         int nb, const int32_t* __restrict__ bij,
                                                         const long long* __restrict__ off,
                                                         int32_t* __restrict__ cbond, int32_t* __restrict__ csamp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int2* bonds = reinterpret_cast<int2*>(smem_raw);
    int8_t* rowbuf = reinterpret_cast<int8_t*>(bonds + nb);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        bool bad = false;
        bonds[b] = checked_bond(bij, b, N, &bad);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int8_t* row = rowbuf + wid * N;
    for (long long s = (long long)blockIdx.x * CONN_WARPS + wid; s < ns; s += (long long)gridDim.x * CONN_WARPS) {
        for (int k = lane; k < N; k += 32) row[k] = x[s * N + k];
        __syncwarp();
        long long pos = off[s];
        for (int b0 = 0; b0 < nb; b0 += 32) {
            const int b = b0 + lane;
            bool anti = false;
            if (b < nb) anti = anti_aligned(row, bonds[b]);
            const unsigned m = __ballot_sync(0xffffffffu, anti);
            if (anti) {
                const long long at = pos + __popc(m & ((1u << lane) - 1u));
                cbond[at] = b;
                csamp[at] = (int32_t)s;
            }
            pos += __popc(m);
        }
        __syncwarp();
    }
}

// Exclusive scan of int32 counts into int64 offsets [ns + 1], one CTA.
__global__ void __launch_bounds__(1024) scan_kernel(const int32_t* __restrict__ cnt, long long ns,
                                                     long long* __restrict__ off) {
    __shared__ long long part[1024];
    const long long per = (ns + blockDim.x - 1) / blockDim.x;
    const long long a = threadIdx.x * per;
    const long long b = (a + per) < ns ? (a + per) : ns;
    long long sum = 0;
    for (long long i = a; i < b; ++i) sum += cnt[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int d = 1; d < (int)blockDim.x; d <<= 1) {
        long long v = (threadIdx.x >= (unsigned)d) ? part[threadIdx.x - d] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    long long run = part[threadIdx.x] - sum;  // exclusive
    for (long long i = a; i < b; ++i) {
        off[i] = run;
        run += cnt[i];
    }
    if (threadIdx.x == blockDim.x - 1) off[ns] = part[threadIdx.x];
}

// Connected-configuration amplitudes ratios: term[c] = 2 c J_b sign exp(ln psi(x') - ln psi(x)).
template <typename R>
__global__ void __launch_bounds__(256) conn_terms_kernel(ModelDesc md, const cx<R>* __restrict__ th,
                                                          const cx<R>* __restrict__ wt,
                                                          const cx<R>* __restrict__ Z,
                                                          const c128* __restrict__ logpsi,
                                                          const int8_t* __restrict__ x, HamDesc h,
                                                          const int32_t* __restrict__ cbond,
                                                          const int32_t* __restrict__ csamp,
                                                          const long long* __restrict__ nconn_ptr, int TR,
                                                          c128* __restrict__ terms) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ld = md.maxw;
    cx<R>* A = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* B = A + (size_t)TR * ld;
    int* ssamp = reinterpret_cast<int*>(B + (size_t)TR * ld);
    int* sbond = ssamp + TR;
    R* sxi = reinterpret_cast<R*>(sbond + TR);
    R* sxj = sxi + TR;
    int* si = reinterpret_cast<int*>(sxj + TR);
    int* sj = si + TR;
    cx<R>* lpn = reinterpret_cast<cx<R>*>(((uintptr_t)(sj + TR) + 15) & ~(uintptr_t)15);
    const long long nconn = *nconn_ptr;  // total connections (device-side scan result)
    const long long c0 = (long long)blockIdx.x * TR;
    if (c0 >= nconn) return;
    const int rows = (int)((nconn - c0) < TR ? (nconn - c0) : TR);
    const int N = md.N;
    for (int r = threadIdx.x; r < TR; r += blockDim.x) {
        if (r < rows) {
            const int s = csamp[c0 + r], b = cbond[c0 + r];
            const int i = h.bond_ij[2 * b], j = h.bond_ij[2 * b + 1];
            ssamp[r] = s;
            sbond[r] = b;
            si[r] = i;
            sj[r] = j;
            sxi[r] = (R)x[(long long)s * N + i];
            sxj[r] = (R)x[(long long)s * N + j];
        } else {
            ssamp[r] = -1;
            sbond[r] = 0;
            si[r] = 0;
            sj[r] = 0;
            sxi[r] = R(0);
            sxj[r] = R(0);
        }
    }
    __syncthreads();
    const int out0 = md.widths[1];
    const cx<R>* W0T = wt + md.wtoff[0];  // [N][out0]
    const bool rbm = md.kind == NQS_RBM;
    const bool linear = (!rbm) && md.L == 1;
    if (!linear) {
        // first layer: z' = z - 2 x_i W[:, i] - 2 x_j W[:, j]
        for (int idx = threadIdx.x; idx < TR * out0; idx += blockDim.x) {
            const int r = idx / out0, u = idx % out0;
            cx<R> v = mk<R>(R(0), R(0));
            if (r < rows) {
                const cx<R> z = Z[md.zoff[0] + (long long)ssamp[r] * out0 + u];
                const cx<R> wi = W0T[(long long)si[r] * out0 + u];
                const cx<R> wj = W0T[(long long)sj[r] * out0 + u];
                const R ai = R(-2) * sxi[r], aj = R(-2) * sxj[r];
                const cx<R> zp = mk<R>(z.re + ai * wi.re + aj * wj.re, z.im + ai * wi.im + aj * wj.im);
                if (rbm) {
                    // difference of the hidden-unit terms
                    v = clncosh(zp) - clncosh(z);
                } else {
                    v = clncosh(zp);
                }
            }
            A[r * ld + u] = v;
        }
        __syncthreads();
    }
    if (rbm) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int r = wid; r < rows; r += nw) {
            cx<R> acc = mk<R>(R(0), R(0));
            for (int u = lane; u < out0; u += 32) acc = acc + A[r * ld + u];
            acc = warp_sum(acc);
            if (lane == 0) {
                const cx<R> ai = th[md.aoff + si[r]], aj = th[md.aoff + sj[r]];
                acc.re += R(-2) * (sxi[r] * ai.re + sxj[r] * aj.re);
                acc.im += R(-2) * (sxi[r] * ai.im + sxj[r] * aj.im);
                lpn[r] = acc;  // ln psi(x') - ln psi(x)
            }
        }
    } else if (linear) {
        for (int r = threadIdx.x; r < rows; r += blockDim.x) {
            const cx<R> wi = th[md.woff[0] + si[r]], wj = th[md.woff[0] + sj[r]];
            lpn[r] = mk<R>(R(-2) * (sxi[r] * wi.re + sxj[r] * wj.re), R(-2) * (sxi[r] * wi.im + sxj[r] * wj.im));
        }
    } else {
        for (int l = 1; l < md.L; ++l) {
            const int out = md.widths[l + 1], in = md.widths[l];
            const cx<R>* W = wt + md.wtoff[l];
            const cx<R>* bias = th + md.boff[l];
            const int groups = (TR / 4) * out;
            const bool last = l == md.L - 1;
            for (int g = threadIdx.x; g < groups; g += blockDim.x) {
                const int rg = g / out, j = g % out;
                cx<R> acc[4];
                const cx<R> bj = bias[j];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = bj;
                for (int k = 0; k < in; ++k) {
                    const cx<R> w = W[(long long)k * out + j];
#pragma unroll
                    for (int q = 0; q < 4; ++q) cmac(acc[q], A[(4 * rg + q) * ld + k], w);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int r = 4 * rg + q;
                    if (last) {
                        if (r < rows) lpn[r] = acc[q];
                    } else {
                        B[r * ld + j] = clncosh(acc[q]);
                    }
                }
            }
            __syncthreads();
            cx<R>* t = A;
            A = B;
            B = t;
        }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        cx<double> d = ccast<double>(lpn[r]);
        if (!rbm && !linear) d = d - logpsi[ssamp[r]];
        const double m = exp(d.re);
        double sn, cs;
        sincos(d.im, &sn, &cs);
        const double f = 2.0 * h.c * h.bond_J[sbond[r]] * (double)h.sign_rule;
        terms[c0 + r] = mk<double>(f * m * cs, f * m * sn);
    }
}

// ------------------------------------------------------------------ double-float hidden layers
// FP64 local energies of FFNNs: the hidden-layer products of the connected forwards run in
// double-float arithmetic (each value an unevaluated sum hi + lo of two FP32 numbers; the
// leading product is made exact with an FMA, cross terms and the TwoSum error go to the low
// word), about 2^-48 relative, on the FP32 units; the first-layer update and ln cosh stay
// in FP64. GB300's FP32 rate is some 64 times its FP64 rate.
struct df2 {
    float rh, ih, rl, il;  // re = rh + rl, im = ih + il
};

__device__ __forceinline__ df2 to_df(c128 z) {
    df2 d;
    d.rh = __double2float_rn(z.re);
    d.rl = __double2float_rn(z.re - (double)d.rh);
    d.ih = __double2float_rn(z.im);
    d.il = __double2float_rn(z.im - (double)d.ih);
    return d;
}

// (ah, al) += (xh + xl)(yh + yl). The intrinsics keep the compiler from contracting the
// error-free transformations into FMAs.
__device__ __forceinline__ void df_mac(float& ah, float& al, float xh, float xl, float yh, float yl) {
    const float ph = __fmul_rn(xh, yh);
    const float pl = fmaf(xh, yl, fmaf(xl, yh, fmaf(xh, yh, -ph)));
    const float s = __fadd_rn(ah, ph);
    const float bb = __fsub_rn(s, ah);
    const float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(ph, bb));
    ah = s;
    al = __fadd_rn(al, __fadd_rn(e, pl));
}

// ---- ln cosh in double-float arithmetic (the hidden units of the connected forwards)
// Building blocks: TwoSum/Fast-TwoSum (Knuth; Dekker 1971) and the FMA-based exact product.
// exp: x = k ln2 + r (ln2 in three parts, the first with 8 trailing zero bits so that k ln2_1
// is exact for |k| < 256), expm1(r 2^-10) by its Taylor series, then ten doublings
// expm1(2y) = expm1(y)(2 + expm1(y)). sin/cos: h = k pi/2 + r (three-part pi/2), Taylor series
// at r/8, three doublings sin 2a = 2 sin a cos a, cos 2a = 1 - 2 sin^2 a, quadrant from k.
// log and atan2: one Newton step from the FP32 value. About 2^-46 relative; the rare
// arguments outside the reductions' ranges take the FP64 ln cosh.
namespace dfm {
struct dff {
    float h, l;
};
__device__ __forceinline__ dff mkf(float h, float l) {
    dff r;
    r.h = h;
    r.l = l;
    return r;
}
__device__ __forceinline__ dff fts(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return mkf(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dff add(dff a, dff b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return fts(s, e);
}
__device__ __forceinline__ dff mul(dff a, dff b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    return fts(p, e);
}
__device__ __forceinline__ dff prodf(float a, float b) {  // exact a b
    const float p = __fmul_rn(a, b);
    return mkf(p, fmaf(a, b, -p));
}
__device__ __forceinline__ dff neg(dff a) { return mkf(-a.h, -a.l); }
__device__ __forceinline__ dff scl(dff a, float s) { return mkf(a.h * s, a.l * s); }  // s a power of two
__device__ __forceinline__ dff from_double(double x) {
    const float h = __double2float_rn(x);
    return mkf(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }  // -126 <= k <= 127

__device__ __forceinline__ dff expm1_core(dff r) {  // |r| <= ln2 / 2
    const dff rs = scl(r, 0x1p-10f);
    dff p = mkf(0x1.111112p-7f, -0x1.dddddep-32f);
    p = add(mul(p, rs), mkf(0x1.555556p-5f, -0x1.555556p-30f));
    p = add(mul(p, rs), mkf(0x1.555556p-3f, -0x1.555556p-28f));
    p = add(mul(p, rs), mkf(0x1p-1f, 0.f));
    p = add(mul(p, rs), mkf(1.f, 0.f));
    dff e = mul(p, rs);
#pragma unroll
    for (int q = 0; q < 10; ++q) e = mul(e, add(mkf(2.f, 0.f), e));
    return e;
}
// reduction x = k ln2 + r (|k| < 256)
__device__ __forceinline__ dff red_ln2(dff x, float k) {
    dff t = mkf(__fsub_rn(x.h, __fmul_rn(k, 0x1.62e4p-1f)), 0.f);
    t = add(t, mkf(x.l, 0.f));
    t = add(t, neg(prodf(k, 0x1.7f7d1cp-20f)));
    return add(t, mkf(-__fmul_rn(k, 0x1.ef357ap-45f), 0.f));
}
// exp(y) for |y| <= 87
__device__ __forceinline__ dff exp_df(dff y) {
    const float k = rintf(y.h * 1.44269504f);
    const dff o = add(mkf(1.f, 0.f), expm1_core(red_ln2(y, k)));
    return scl(o, pow2f((int)k));
}
// rho = exp(x) and om = 1 - rho for x <= 0
__device__ __forceinline__ void exp_om(dff x, dff* rho, dff* om) {
    if (x.h < -60.f) {
        *rho = mkf(0.f, 0.f);
        *om = mkf(1.f, 0.f);
        return;
    }
    const float k = rintf(x.h * 1.44269504f);
    const dff e = expm1_core(red_ln2(x, k));
    *rho = scl(add(mkf(1.f, 0.f), e), pow2f((int)k));
    *om = (k == 0.f) ? neg(e) : add(mkf(1.f, 0.f), neg(*rho));
}
// (sin h, cos h) for |h| < 256 pi/2
__device__ __forceinline__ void sincos_df(dff h, dff* sn, dff* cs) {
    const float k = rintf(h.h * 0.636619772f);
    dff t = mkf(__fsub_rn(h.h, __fmul_rn(k, 0x1.922p+0f)), 0.f);
    t = add(t, mkf(h.l, 0.f));
    t = add(t, neg(prodf(k, -0x1.2aeef4p-18f)));
    t = add(t, mkf(-__fmul_rn(k, -0x1.73dcb4p-43f), 0.f));
    const dff rs = scl(t, 0.125f);
    const dff x2 = mul(rs, rs);
    dff p = mkf(0x1.71de3ap-19f, 0x1.55b1ccp-45f);
    p = add(mul(p, x2), mkf(-0x1.a01a02p-13f, 0x1.7f97fap-39f));
    p = add(mul(p, x2), mkf(0x1.111112p-7f, -0x1.dddddep-32f));
    p = add(mul(p, x2), mkf(-0x1.555556p-3f, 0x1.555556p-28f));
    p = add(mul(p, x2), mkf(1.f, 0.f));
    dff s = mul(p, rs);
    dff c = mkf(-0x1.27e4fcp-22f, 0x1.10ec14p-47f);
    c = add(mul(c, x2), mkf(0x1.a01a02p-16f, -0x1.7f97fap-42f));
    c = add(mul(c, x2), mkf(-0x1.6c16c2p-10f, 0x1.27d27ep-35f));
    c = add(mul(c, x2), mkf(0x1.555556p-5f, -0x1.555556p-30f));
    c = add(mul(c, x2), mkf(-0x1p-1f, 0.f));
    c = add(mul(c, x2), mkf(1.f, 0.f));
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const dff s2 = scl(mul(s, c), 2.f);
        c = add(mkf(1.f, 0.f), scl(mul(s, s), -2.f));
        s = s2;
    }
    switch (((int)k) & 3) {
        case 0: *sn = s; *cs = c; break;
        case 1: *sn = c; *cs = neg(s); break;
        case 2: *sn = neg(s); *cs = neg(c); break;
        default: *sn = neg(c); *cs = s; break;
    }
}
__device__ __forceinline__ dff log_df(dff x) {  // x > 1e-30
    const float y0 = logf(x.h);
    return add(mkf(y0, 0.f), add(mul(x, exp_df(mkf(-y0, 0.f))), mkf(-1.f, 0.f)));
}
__device__ __forceinline__ dff atan2_df(dff Y, dff X) {  // X >= 0
    const float th = atan2f(Y.h, X.h);
    dff s, c;
    sincos_df(mkf(th, 0.f), &s, &c);
    const dff num = add(mul(Y, c), neg(mul(X, s)));
    const float den = fmaf(X.h, c.h, Y.h * s.h);
    return den != 0.f ? add(mkf(th, 0.f), mkf(num.h / den, 0.f)) : mkf(th, 0.f);
}
// ln cosh(zr + i zi), same branch as clncosh; false when the argument is outside the
// ranges above (the caller then takes the FP64 ln cosh).
__device__ __forceinline__ bool lncosh_df(dff zr, dff zi, dff* re, dff* im) {
    if (!(fabsf(zi.h) < 400.f)) return false;
    const float s = zr.h >= 0.f ? 1.f : -1.f;
    const dff ax = scl(zr, s), h = scl(zi, -s);
    dff sh, ch, rho, om;
    sincos_df(h, &sh, &ch);
    exp_om(scl(ax, -2.f), &rho, &om);
    const dff rc2 = mul(rho, mul(ch, ch));
    const dff mod2 = add(mul(om, om), scl(rc2, 4.f));
    if (!(mod2.h > 1e-30f)) return false;
    const dff lr = scl(log_df(mod2), 0.5f);
    const dff li = atan2_df(mul(rho, scl(mul(sh, ch), 2.f)), add(om, scl(rc2, 2.f)));
    *re = add(add(ax, mkf(-0x1.62e43p-1f, 0x1.05c61p-29f)), lr);
    *im = add(scl(zi, s), li);
    return true;
}
}  // namespace dfm

// ln cosh of a double-float complex value into the shared-memory layout
__device__ __forceinline__ df2 lncosh_to_df2(dfm::dff zr, dfm::dff zi) {
    dfm::dff re, im;
    if (dfm::lncosh_df(zr, zi, &re, &im)) {
        df2 d;
        d.rh = re.h;
        d.rl = re.l;
        d.ih = im.h;
        d.il = im.l;
        return d;
    }
    return to_df(clncosh(mk<double>((double)zr.h + (double)zr.l, (double)zi.h + (double)zi.l)));
}

__global__ void split_weights_kernel(const c128* __restrict__ w, long long n, float4* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const df2 d = to_df(w[i]);
        out[i] = make_float4(d.rh, d.ih, d.rl, d.il);
    }
}

__global__ void __launch_bounds__(256) conn_terms_df_kernel(ModelDesc md, const c128* __restrict__ th,
                                                             const c128* __restrict__ wt,
                                                             const float4* __restrict__ wdf,
                                                             const c128* __restrict__ Z,
                                                             const c128* __restrict__ logpsi,
                                                             const int8_t* __restrict__ x, HamDesc h,
                                                             const int32_t* __restrict__ cbond,
                                                             const int32_t* __restrict__ csamp,
                                                             const long long* __restrict__ nconn_ptr,
                                                             const long long* __restrict__ cidx, int TR,
                                                             c128* __restrict__ terms) {
    // cidx (optional): the rows are connections cidx[0 .. *nconn_ptr) instead of 0 .. *nconn_ptr
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ld = md.maxw;
    df2* const A0 = reinterpret_cast<df2*>(smem_raw);
    df2* const B0 = A0 + (size_t)TR * ld;
    int* ssamp = reinterpret_cast<int*>(B0 + (size_t)TR * ld);
    int* sbond = ssamp + TR;
    double* sxi = reinterpret_cast<double*>(sbond + TR);
    double* sxj = sxi + TR;
    int* si = reinterpret_cast<int*>(sxj + TR);
    int* sj = si + TR;
    c128* lpn = reinterpret_cast<c128*>(((uintptr_t)(sj + TR) + 15) & ~(uintptr_t)15);
    const long long nconn = *nconn_ptr;
    const int N = md.N;
    // grid-stride over tiles of TR rows (the grid may be smaller than the list)
    for (long long c0 = (long long)blockIdx.x * TR; c0 < nconn; c0 += (long long)gridDim.x * TR) {
    df2* A = A0;
    df2* B = B0;
    const int rows = (int)((nconn - c0) < TR ? (nconn - c0) : TR);
    for (int r = threadIdx.x; r < TR; r += blockDim.x) {
        if (r < rows) {
            const long long c = cidx ? cidx[c0 + r] : c0 + r;
            const int s = csamp[c], b = cbond[c];
            const int i = h.bond_ij[2 * b], j = h.bond_ij[2 * b + 1];
            ssamp[r] = s;
            sbond[r] = b;
            si[r] = i;
            sj[r] = j;
            sxi[r] = (double)x[(long long)s * N + i];
            sxj[r] = (double)x[(long long)s * N + j];
        } else {
            ssamp[r] = -1;
            sbond[r] = 0;
            si[r] = 0;
            sj[r] = 0;
            sxi[r] = 0.0;
            sxj[r] = 0.0;
        }
    }
    __syncthreads();
    // first layer in FP64: z' = z - 2 x_i W[:, i] - 2 x_j W[:, j], then ln cosh
    const int out0 = md.widths[1];
    const c128* W0T = wt + md.wtoff[0];  // [N][out0]
    for (int idx = threadIdx.x; idx < TR * out0; idx += blockDim.x) {
        const int r = idx / out0, u = idx % out0;
        c128 v = mk<double>(0.0, 0.0);
        if (r < rows) {
            const c128 z = Z[md.zoff[0] + (long long)ssamp[r] * out0 + u];
            const c128 wi = W0T[(long long)si[r] * out0 + u];
            const c128 wj = W0T[(long long)sj[r] * out0 + u];
            const double ai = -2.0 * sxi[r], aj = -2.0 * sxj[r];
            v = mk<double>(z.re + ai * wi.re + aj * wj.re, z.im + ai * wi.im + aj * wj.im);
        }
        A[r * ld + u] = r < rows ? lncosh_to_df2(dfm::from_double(v.re), dfm::from_double(v.im)) : to_df(v);
    }
    __syncthreads();
    for (int l = 1; l < md.L; ++l) {
        const int out = md.widths[l + 1], in = md.widths[l];
        const float4* W = wdf + md.wtoff[l];
        const c128* bias = th + md.boff[l];
        const int groups = (TR / 4) * out;
        const bool last = l == md.L - 1;
        for (int g = threadIdx.x; g < groups; g += blockDim.x) {
            const int rg = g / out, j = g % out;
            df2 acc[4];
            const df2 bj = to_df(bias[j]);
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = bj;
            for (int k = 0; k < in; ++k) {
                const float4 w = W[(long long)k * out + j];  // (re hi, im hi, re lo, im lo)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const df2 a = A[(4 * rg + q) * ld + k];
                    df_mac(acc[q].rh, acc[q].rl, a.rh, a.rl, w.x, w.z);    // + a_re w_re
                    df_mac(acc[q].rh, acc[q].rl, -a.ih, -a.il, w.y, w.w);  // - a_im w_im
                    df_mac(acc[q].ih, acc[q].il, a.rh, a.rl, w.y, w.w);    // + a_re w_im
                    df_mac(acc[q].ih, acc[q].il, a.ih, a.il, w.x, w.z);    // + a_im w_re
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = 4 * rg + q;
                if (last) {
                    if (r < rows)
                        lpn[r] = mk<double>((double)acc[q].rh + (double)acc[q].rl,
                                            (double)acc[q].ih + (double)acc[q].il);
                } else {
                    // renormalise the accumulated pair before ln cosh
                    const dfm::dff zr = dfm::fts(acc[q].rh, acc[q].rl), zi = dfm::fts(acc[q].ih, acc[q].il);
                    B[r * ld + j] = lncosh_to_df2(zr, zi);
                }
            }
        }
        __syncthreads();
        df2* t = A;
        A = B;
        B = t;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const c128 d = lpn[r] - logpsi[ssamp[r]];
        const double m = exp(d.re);
        double sn, cs;
        sincos(d.im, &sn, &cs);
        const double f = 2.0 * h.c * h.bond_J[sbond[r]] * (double)h.sign_rule;
        terms[cidx ? cidx[c0 + r] : c0 + r] = mk<double>(f * m * cs, f * m * sn);
    }
    __syncthreads();
    }
}

// ------------------------------------------------------------------ FP32 difference propagation
// Local energies of FFNNs in the split precisions. Rather than pushing every connected
// configuration x' through the network, the kernel propagates its differences to the parent
// sample x: the first layer changes by dz = -2 x_i W[:, i] - 2 x_j W[:, j] (the bias cancels),
// every hidden layer by
//   dh = lncosh(z + dz) - lncosh(z) = log1p(w),
//   w  = cosh(z + dz) / cosh(z) - 1 = 2 sinh(dz/2) (sinh(dz/2) + cosh(dz/2) tanh z),
// (from cosh(z + dz) = cosh z cosh dz + sinh z sinh dz), the next pre-activation by W dh, and
// ln psi(x') - ln psi(x) = W_L dh. The FP32 roundings then act on the differences, not on
// the activations and ln psi, which are larger. z and tanh z come from the parent's FP64
// forward. Re log1p(w) = ln|cosh z' / cosh z| has no branch; the imaginary part has to follow
// the ln cosh branch of the exact forward (s = sign Re z), which differs from log1p's
// principal value by 2 pi k. With s' = s, |Im dz| < 1/2 and |Im log1p w| < 5/2, k = 0
// (each ln cosh is s Im z plus an angle in [-pi/2, pi/2], so the exact difference is within
// pi + 1/2 of 0); otherwise k is taken from FP32 values of both ln cosh. A connection goes to
// a list for the double-float kernel when FP32 cannot follow the exact forward: Re z' within
// rounding of 0 while |Im z'| > 1.5 (there ln cosh jumps by 2 pi i), |1 + w| < 1e-3 (ln of
// a near-zero cosh), or arguments outside the ranges of the FP32 functions.
constexpr int DP_WARPS = 8;

// (z, tanh z) of every hidden unit of the parent samples, FP32 copies of the FP64 forward
__global__ void dp_parent_kernel(ModelDesc md, const c128* __restrict__ Z, long long ns, float4* __restrict__ pz) {
    for (int l = 0; l + 1 < md.L; ++l) {
        const long long n = ns * md.widths[l + 1];
        const c128* z = Z + md.zoff[l];
        float4* p = pz + md.zoff[l];
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
             e += (long long)gridDim.x * blockDim.x) {
            const c128 v = z[e];
            const c128 t = ctanh(v);
            p[e] = make_float4((float)v.re, (float)v.im, (float)t.re, (float)t.im);
        }
    }
}

__global__ void weights_f32_kernel(const c128* __restrict__ w, long long n, float2* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = make_float2((float)w[i].re, (float)w[i].im);
}

// dh of one hidden unit; p = (Re z, Im z, Re tanh z, Im tanh z) of the parent. *bad: the
// connection needs the exact kernel.
__device__ __forceinline__ float2 dp_lncosh_diff(float2 dz, float4 p, bool* bad) {
    const float zr = p.x + dz.x, zi = p.y + dz.y;  // z' = z + dz
    if (!(fabsf(dz.x) < 40.f && fabsf(dz.y) < 1e4f && p.z * p.z + p.w * p.w < 1e8f) ||
        (fabsf(zr) < 2e-4f + 1e-5f * (fabsf(p.x) + fabsf(dz.x)) && fabsf(zi) > 1.5f)) {
        *bad = true;
        return make_float2(0.f, 0.f);
    }
    float sb, cb;
    sincosf(0.5f * dz.y, &sb, &cb);
    const float sa = sinhf(0.5f * dz.x), ca = coshf(0.5f * dz.x);
    const float shr = sa * cb, shi = ca * sb;  // sinh(dz/2)
    const float chr = ca * cb, chi = sa * sb;  // cosh(dz/2)
    const float qr = shr + (chr * p.z - chi * p.w), qi = shi + (chr * p.w + chi * p.z);
    const float wr = 2.f * (shr * qr - shi * qi), wi = 2.f * (shr * qi + shi * qr);
    const float ar = 1.f + wr;
    const float mod2 = ar * ar + wi * wi;  // |1 + w|^2
    if (!(mod2 > 1e-6f)) {
        *bad = true;
        return make_float2(0.f, 0.f);
    }
    const float re = mod2 > 0.25f ? 0.5f * log1pf(fmaf(wr, wr, fmaf(wi, wi, 2.f * wr))) : 0.5f * logf(mod2);
    float im = atan2f(wi, ar);
    if ((zr >= 0.f) != (p.x >= 0.f) || fabsf(dz.y) >= 0.5f || fabsf(im) >= 2.5f) {
        const float i1 = clncosh(mk<float>(zr, zi)).im, i0 = clncosh(mk<float>(p.x, p.y)).im;
        im = fmaf(rintf((i1 - i0 - im) * 0.159154943f), 6.28318531f, im);
    }
    return make_float2(re, im);
}

// B[r][c] = sum_k A[r][k] W[k][c] for the RPW rows of this warp; lanes own columns c and c + 32
// of every 64-column pass. A in shared memory (broadcast reads), W^T [in][out] from L1/L2.
template <int RPW>
__device__ __forceinline__ void dp_matvec(const float2* __restrict__ A, float2* __restrict__ B, int ld,
                                          const float2* __restrict__ W, int in, int out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = warp * RPW;
    for (int cb = 0; cb < out; cb += 64) {
        const int c0 = cb + lane, c1 = cb + 32 + lane;
        const bool v0 = c0 < out, v1 = c1 < out;
        float2 a0[RPW], a1[RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q) a0[q] = a1[q] = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int k = 0; k < in; ++k) {
            const float2 w0 = v0 ? __ldg(&W[(long long)k * out + c0]) : make_float2(0.f, 0.f);
            const float2 w1 = v1 ? __ldg(&W[(long long)k * out + c1]) : make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < RPW; ++q) {
                const float2 a = A[(r0 + q) * ld + k];
                a0[q].x = fmaf(a.x, w0.x, fmaf(-a.y, w0.y, a0[q].x));
                a0[q].y = fmaf(a.x, w0.y, fmaf(a.y, w0.x, a0[q].y));
                a1[q].x = fmaf(a.x, w1.x, fmaf(-a.y, w1.y, a1[q].x));
                a1[q].y = fmaf(a.x, w1.y, fmaf(a.y, w1.x, a1[q].y));
            }
        }
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            if (v0) B[(r0 + q) * ld + c0] = a0[q];
            if (v1) B[(r0 + q) * ld + c1] = a1[q];
        }
    }
}

// One tile of DP_WARPS * RPW connections per CTA; two [TR][ld] FP32 complex buffers in shared
// memory (ld = widest hidden layer). Connections it cannot follow go to fb_list.
template <int RPW>
__global__ void __launch_bounds__(256) conn_terms_dp_kernel(ModelDesc md, const float2* __restrict__ w32,
                                                             const float4* __restrict__ pz,
                                                             const int8_t* __restrict__ x, HamDesc h,
                                                             const int32_t* __restrict__ cbond,
                                                             const int32_t* __restrict__ csamp,
                                                             const long long* __restrict__ nconn_ptr, int ld,
                                                             c128* __restrict__ terms, long long* __restrict__ fb_list,
                                                             unsigned long long* __restrict__ fb_count, int fb_all) {
    constexpr int TR = DP_WARPS * RPW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* D = reinterpret_cast<float2*>(smem_raw);  // dz of the current layer, then dh in place
    float2* E = D + (size_t)TR * ld;                   // dz of the next layer
    __shared__ int ssamp[TR], sbond[TR], si[TR], sj[TR], sflag[TR];
    __shared__ float sxi[TR], sxj[TR];
    __shared__ float2 sd[TR];
    const long long nconn = *nconn_ptr;
    const long long c0 = (long long)blockIdx.x * TR;
    if (c0 >= nconn) return;
    const int rows = (int)((nconn - c0) < TR ? (nconn - c0) : TR);
    const int N = md.N;
    for (int r = threadIdx.x; r < TR; r += blockDim.x) {
        int s = 0, b = 0, i = 0, j = 0;
        float xi = 0.f, xj = 0.f;
        if (r < rows) {  // rows past the end repeat sample 0 with zero spins and are not written
            s = csamp[c0 + r];
            b = cbond[c0 + r];
            i = h.bond_ij[2 * b];
            j = h.bond_ij[2 * b + 1];
            xi = (float)x[(long long)s * N + i];
            xj = (float)x[(long long)s * N + j];
        }
        ssamp[r] = s;
        sbond[r] = b;
        si[r] = i;
        sj[r] = j;
        sxi[r] = xi;
        sxj[r] = xj;
        sflag[r] = 0;
    }
    __syncthreads();
    {  // first layer: dz = -2 x_i W[:, i] - 2 x_j W[:, j] (one rounding)
        const int out0 = md.widths[1];
        const float2* W0 = w32 + md.wtoff[0];  // [N][out0]
        for (int idx = threadIdx.x; idx < TR * out0; idx += blockDim.x) {
            const int r = idx / out0, u = idx - r * out0;
            const float2 wi = W0[(long long)si[r] * out0 + u], wj = W0[(long long)sj[r] * out0 + u];
            const float ai = -2.f * sxi[r], aj = -2.f * sxj[r];
            D[r * ld + u] = make_float2(fmaf(ai, wi.x, aj * wj.x), fmaf(ai, wi.y, aj * wj.y));
        }
    }
    __syncthreads();
    for (int l = 0; l + 1 < md.L; ++l) {
        const int out = md.widths[l + 1];
        const float4* P = pz + md.zoff[l];
        for (int idx = threadIdx.x; idx < TR * out; idx += blockDim.x) {
            const int r = idx / out, u = idx - r * out;
            bool bad = false;
            const float2 dh = dp_lncosh_diff(D[r * ld + u], P[(long long)ssamp[r] * out + u], &bad);
            if (bad) sflag[r] = 1;
            D[r * ld + u] = dh;
        }
        __syncthreads();
        const int nout = md.widths[l + 2];
        const float2* Wn = w32 + md.wtoff[l + 1];  // [out][nout]
        if (l + 2 == md.L) {  // output layer (one unit): a dot product per row
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            for (int q = 0; q < RPW; ++q) {
                const int r = warp * RPW + q;
                float re = 0.f, im = 0.f;
                for (int k = lane; k < out; k += 32) {
                    const float2 a = D[r * ld + k], w = __ldg(&Wn[k]);
                    re = fmaf(a.x, w.x, fmaf(-a.y, w.y, re));
                    im = fmaf(a.x, w.y, fmaf(a.y, w.x, im));
                }
                re = warp_sum(re);
                im = warp_sum(im);
                if (lane == 0) sd[r] = make_float2(re, im);
            }
        } else {
            dp_matvec<RPW>(D, E, ld, Wn, out, nout);
            float2* t = D;
            D = E;
            E = t;
        }
        __syncthreads();
    }
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const long long c = c0 + r;
        const float2 d = sd[r];  // ln psi(x') - ln psi(x)
        if (fb_all || sflag[r] || !(fabsf(d.x) < 80.f) || !(fabsf(d.y) < 1e6f)) {
            fb_list[atomicAdd(fb_count, 1ull)] = c;
        } else {
            const double m = exp((double)d.x);
            double sn, cs;
            sincos((double)d.y, &sn, &cs);
            const double f = 2.0 * h.c * h.bond_J[sbond[r]] * (double)h.sign_rule;
            terms[c] = mk<double>(f * m * cs, f * m * sn);
        }
    }
}

__global__ void eloc_reduce_kernel(const int8_t* __restrict__ x, long long ns, HamDesc h,
                                   const long long* __restrict__ off, const c128* __restrict__ terms,
                                   c128* __restrict__ eloc, DevStatus* status) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= ns) return;
    double diag = 0.0;
    const int8_t* row = x + s * h.n_sites;
    for (int b = 0; b < h.n_bonds; ++b) {
        const int i = h.bond_ij[2 * b], j = h.bond_ij[2 * b + 1];
        // a bad bond was reported by conn_count_kernel; it contributes nothing here
        if (i < 0 || i >= h.n_sites || j < 0 || j >= h.n_sites || i == j) continue;
        diag += h.bond_J[b] * (double)(row[i] * row[j]);
    }
    c128 e = mk<double>(h.c * diag, 0.0);
    for (long long c = off[s]; c < off[s + 1]; ++c) e = e + terms[c];
    if (!finite_cx(e)) set_status(status, NQS_ERR_NONFINITE, W_ELOC, s);
    eloc[s] = e;
}

// ------------------------------------------------------------------ launchers
static size_t conn_smem(const HamDesc& h) {
    return (size_t)h.n_bonds * sizeof(int2) + (size_t)CONN_WARPS * h.n_sites + 16;
}
static int conn_grid(long long ns) {
    long long g = (ns + CONN_WARPS - 1) / CONN_WARPS;
    return (int)(g < 8192 ? (g < 1 ? 1 : g) : 8192);
}

cudaError_t launch_conn_count(const int8_t* x, long long ns, const HamDesc& h, int32_t* cnt, DevStatus* status,
                              cudaStream_t st) {
    if (ns <= 0) return cudaSuccess;
    const size_t sm = conn_smem(h);
    cudaError_t e = cudaFuncSetAttribute(conn_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    count_launch();
    conn_count_kernel<<<conn_grid(ns), 32 * CONN_WARPS, sm, st>>>(x, ns, h.n_sites, h.n_bonds, h.bond_ij, cnt,
                                                                  status);
    return cudaGetLastError();
}
cudaError_t launch_scan(const int32_t* cnt, long long ns, long long* off, cudaStream_t st) {
    count_launch();
    scan_kernel<<<1, 1024, 0, st>>>(cnt, ns, off);
    return cudaGetLastError();
}
cudaError_t launch_conn_fill(const int8_t* x, long long ns, const HamDesc& h, const long long* off,
                             int32_t* conn_bond, int32_t* conn_sample, cudaStream_t st) {
    if (ns <= 0) return cudaSuccess;
    const size_t sm = conn_smem(h);
    cudaError_t e = cudaFuncSetAttribute(conn_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    count_launch();
    conn_fill_kernel<<<conn_grid(ns), 32 * CONN_WARPS, sm, st>>>(x, ns, h.n_sites, h.n_bonds, h.bond_ij, off,
                                                                 conn_bond, conn_sample);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t conn_terms_t(const ModelDesc& md, const void* thR, const void* wtR, const void* Z,
                                const c128* logpsi, const int8_t* x, const HamDesc& h,
                                const int32_t* cb, const int32_t* cs, const long long* nconn_ptr,
                                long long max_conn, c128* terms, cudaStream_t st) {
    if (max_conn <= 0) return cudaSuccess;
    long long tr = 180000LL / (2LL * md.maxw * (long long)sizeof(cx<R>));
    tr = tr > 32 ? 32 : tr;
    tr = (tr / 4) * 4;
    const int TR = tr < 4 ? 4 : (int)tr;
    const size_t smem = 2ull * TR * md.maxw * sizeof(cx<R>) + (size_t)TR * (4 * sizeof(int) + 2 * sizeof(R)) +
                        16 + (size_t)TR * sizeof(cx<R>);
    cudaError_t e = cudaFuncSetAttribute(conn_terms_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long grid = (max_conn + TR - 1) / TR;
    count_launch();
    conn_terms_kernel<R><<<(unsigned)grid, 256, smem, st>>>(md, (const cx<R>*)thR, (const cx<R>*)wtR,
                                                            (const cx<R>*)Z, logpsi, x, h, cb, cs, nconn_ptr, TR,
                                                            terms);
    return cudaGetLastError();
}

cudaError_t launch_split_weights(const ModelDesc& md, const void* wtR, void* wdf, cudaStream_t st) {
    const long long n = model_wt_elems(md);
    if (n <= 0) return cudaSuccess;
    count_launch();
    split_weights_kernel<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, st>>>(
        (const c128*)wtR, n, (float4*)wdf);
    return cudaGetLastError();
}

cudaError_t launch_conn_terms(int prec, const ModelDesc& md, const void* thR, const void* wtR, const void* wdf,
                              const void* Z, const c128* logpsi, const int8_t* x, const HamDesc& h,
                              const int32_t* conn_bond, const int32_t* conn_sample,
                              const long long* nconn_ptr, long long max_conn, c128* terms, cudaStream_t st) {
    if (md.kind == NQS_VIT)
        return prec == NQS_FP64 ? launch_vit_conn_terms(md, (const c128*)thR, logpsi, x, h, conn_bond, conn_sample,
                                                        nconn_ptr, max_conn, terms, st)
                                : cudaErrorNotSupported;
    if (prec == NQS_FP64 && md.kind == NQS_FFNN && md.L >= 2 && wdf) {
        if (max_conn <= 0) return cudaSuccess;
        long long tr = 180000LL / (2LL * md.maxw * (long long)sizeof(c128));
        tr = tr > 32 ? 32 : tr;
        tr = (tr / 4) * 4;
        const int TR = tr < 4 ? 4 : (int)tr;
        const size_t smem = 2ull * TR * md.maxw * sizeof(c128) + (size_t)TR * (4 * sizeof(int) + 2 * sizeof(double)) +
                            16 + (size_t)TR * sizeof(c128);
        cudaError_t e =
            cudaFuncSetAttribute(conn_terms_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const long long grid = (max_conn + TR - 1) / TR;
        count_launch();
        conn_terms_df_kernel<<<(unsigned)grid, 256, smem, st>>>(md, (const c128*)thR, (const c128*)wtR,
                                                                 (const float4*)wdf, (const c128*)Z, logpsi, x, h,
                                                                 conn_bond, conn_sample, nconn_ptr, nullptr, TR,
                                                                 terms);
        return cudaGetLastError();
    }
    return prec == NQS_FP64
               ? conn_terms_t<double>(md, thR, wtR, Z, logpsi, x, h, conn_bond, conn_sample, nconn_ptr, max_conn,
                                      terms, st)
               : conn_terms_t<float>(md, thR, wtR, Z, logpsi, x, h, conn_bond, conn_sample, nconn_ptr, max_conn,
                                     terms, st);
}

bool dp_applicable(const ModelDesc& md) {
    if (md.kind != NQS_FFNN || md.L < 2 || md.widths[md.L] != 1) return false;
    return dp_width(md) <= 512;
}
int dp_width(const ModelDesc& md) {
    int w = 0;
    for (int l = 1; l < md.L; ++l) w = md.widths[l] > w ? md.widths[l] : w;
    return w;
}

cudaError_t launch_conn_terms_dp(const ModelDesc& md, const void* thR, const void* wtR, const void* wdf,
                                 const void* Z, const c128* logpsi, const int8_t* x, long long ns, const HamDesc& h,
                                 const int32_t* conn_bond, const int32_t* conn_sample, const long long* nconn_ptr,
                                 long long max_conn, c128* terms, const DpBufs& b, cudaStream_t st) {
    if (max_conn <= 0) return cudaSuccess;
    const long long we = model_wt_elems(md);
    count_launch();
    weights_f32_kernel<<<(unsigned)((we + 255) / 256 < 1024 ? (we + 255) / 256 : 1024), 256, 0, st>>>(
        (const c128*)wtR, we, b.w32);
    count_launch();
    dp_parent_kernel<<<1024, 256, 0, st>>>(md, (const c128*)Z, ns, b.pz);
    cudaError_t e = cudaMemsetAsync(b.fb_count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    // rows per warp: two [TR][ld] FP32 complex buffers within 96 KB (two CTAs per SM)
    const int ld = dp_width(md);
    const int rpw = ld <= 96 ? 8 : (ld <= 192 ? 4 : (ld <= 384 ? 2 : 1));
    const int TR = DP_WARPS * rpw;
    const size_t smem = 2ull * TR * ld * sizeof(float2);
    const long long grid = (max_conn + TR - 1) / TR;
    const int fb_all = dp_fallback_all() ? 1 : 0;
    count_launch();
#define NQS_DP_LAUNCH(R)                                                                                     \
    do {                                                                                                     \
        e = cudaFuncSetAttribute(conn_terms_dp_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                 (int)smem);                                                                 \
        if (e != cudaSuccess) return e;                                                                      \
        conn_terms_dp_kernel<R><<<(unsigned)grid, 256, smem, st>>>(md, b.w32, b.pz, x, h, conn_bond,         \
                                                                   conn_sample, nconn_ptr, ld, terms,       \
                                                                   b.fb_list, b.fb_count, fb_all);          \
    } while (0)
    if (rpw == 8) NQS_DP_LAUNCH(8);
    else if (rpw == 4) NQS_DP_LAUNCH(4);
    else if (rpw == 2) NQS_DP_LAUNCH(2);
    else NQS_DP_LAUNCH(1);
#undef NQS_DP_LAUNCH
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the listed connections in double-float (every CTA past the list's end returns at once)
    e = launch_split_weights(md, wtR, const_cast<void*>(wdf), st);
    if (e != cudaSuccess) return e;
    long long tr = 180000LL / (2LL * md.maxw * (long long)sizeof(c128));
    tr = tr > 32 ? 32 : tr;
    tr = (tr / 4) * 4;
    const int TRf = tr < 4 ? 4 : (int)tr;
    const size_t smf = 2ull * TRf * md.maxw * sizeof(c128) + (size_t)TRf * (4 * sizeof(int) + 2 * sizeof(double)) +
                       16 + (size_t)TRf * sizeof(c128);
    e = cudaFuncSetAttribute(conn_terms_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf);
    if (e != cudaSuccess) return e;
    count_launch();
    const long long tiles = (max_conn + TRf - 1) / TRf;
    conn_terms_df_kernel<<<(unsigned)(tiles < 1024 ? tiles : 1024), 256, smf, st>>>(
        md, (const c128*)thR, (const c128*)wtR, (const float4*)wdf, (const c128*)Z, logpsi, x, h, conn_bond,
        conn_sample, reinterpret_cast<const long long*>(b.fb_count), b.fb_list, TRf, terms);
    return cudaGetLastError();
}

cudaError_t launch_eloc_reduce(const int8_t* x, long long ns, const HamDesc& h, const long long* off,
                               const c128* terms, c128* eloc, DevStatus* status, cudaStream_t st) {
    if (ns <= 0) return cudaSuccess;
    count_launch();
    eloc_reduce_kernel<<<(unsigned)((ns + 127) / 128), 128, 0, st>>>(x, ns, h, off, terms, eloc, status);
    return cudaGetLastError();
}

}  // namespace nqs
