// The transformer wavefunction whose modules give the block partition of Sec. 2 (patching and
// embedding, encoder layers, output layer). The paper leaves the network unspecified; this is
// a holomorphic variant (complex parameters, position-only attention, ln cosh MLP, residuals):
//   h_t = W_E x_t + b_E                             (token t = spins t p .. t p + p - 1)
//   encoder: v_s = W_V h_s; u_t = h_t + sum_s A_ts v_s; z_t = W_1 u_t + b_1;
//            h_t <- u_t + W_2 lncosh(z_t) + b_2
//   ln psi = w_O . sum_t lncosh(h_t) + b_O
// O = d ln psi / d theta by back-propagation through these formulas (plain transposes).
//
// One CTA per configuration: token activations live in shared memory; the forward saves
// h_0 and, per encoder layer, (v, u, z, h_{l+1}) for the Jacobian (Z: [n_s][vsave]). FP64
// throughout. The Jacobian CTA writes its sample's column of the parameter-major O.
#include "internal.cuh"

namespace nqs {
namespace {

constexpr int VT = 128;

__device__ __forceinline__ long long enc_base(const ModelDesc& md, int l) {
    return (long long)md.vd * md.vp + md.vd + (long long)l * md.vE;
}
// saved activations of one sample: h_0 at 0, layer l's v, u, z, h_{l+1} from lay_base(l)
__device__ __forceinline__ long long lay_base(const ModelDesc& md, int l) {
    return (long long)md.vT * md.vd + (long long)l * (3LL * md.vT * md.vd + (long long)md.vT * md.vh);
}
__device__ __forceinline__ long long h_out(const ModelDesc& md, int l) {  // h_{l+1}
    return lay_base(md, l) + 2LL * md.vT * md.vd + (long long)md.vT * md.vh;
}

// Forward of the configuration xs (shared memory) by the whole CTA; H, V, U [T][d] and AZ
// [T][h] are shared scratch; `save` (or NULL) receives the activations. Returns ln psi.
__device__ c128 vit_forward_cta(const ModelDesc& md, const c128* __restrict__ th, const float* xs, c128* H, c128* V,
                                c128* U, c128* AZ, c128* save, double* sh) {
    const int T = md.vT, p = md.vp, d = md.vd, h = md.vh;
    const c128* WE = th;
    const c128* bE = th + (long long)d * p;
    for (int e = threadIdx.x; e < T * d; e += blockDim.x) {
        const int t = e / d, k = e - t * d;
        c128 acc = bE[k];
        for (int j = 0; j < p; ++j) {
            const double xv = xs[t * p + j];
            const c128 w = WE[(long long)k * p + j];
            acc.re = fma(w.re, xv, acc.re);
            acc.im = fma(w.im, xv, acc.im);
        }
        H[e] = acc;
        if (save) save[e] = acc;
    }
    __syncthreads();
    for (int l = 0; l < md.L; ++l) {
        const c128* A = th + enc_base(md, l);
        const c128* WV = A + (long long)T * T;
        const c128* W1 = WV + (long long)d * d;
        const c128* b1 = W1 + (long long)h * d;
        const c128* W2 = b1 + h;
        const c128* b2 = W2 + (long long)d * h;
        c128* sv = save ? save + lay_base(md, l) : nullptr;
        for (int e = threadIdx.x; e < T * d; e += blockDim.x) {  // v = W_V h
            const int t = e / d, k = e - t * d;
            c128 acc = mk<double>(0.0, 0.0);
            for (int j = 0; j < d; ++j) cmac(acc, WV[(long long)k * d + j], H[t * d + j]);
            V[e] = acc;
            if (sv) sv[e] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < T * d; e += blockDim.x) {  // u = h + A v
            const int t = e / d, k = e - t * d;
            c128 acc = H[e];
            for (int s = 0; s < T; ++s) cmac(acc, A[(long long)t * T + s], V[s * d + k]);
            U[e] = acc;
            if (sv) sv[T * d + e] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < T * h; e += blockDim.x) {  // z = W_1 u + b_1, a = lncosh z
            const int t = e / h, m = e - t * h;
            c128 acc = b1[m];
            for (int k = 0; k < d; ++k) cmac(acc, W1[(long long)m * d + k], U[t * d + k]);
            if (sv) sv[2 * T * d + e] = acc;
            AZ[e] = clncosh(acc);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < T * d; e += blockDim.x) {  // h = u + W_2 a + b_2
            const int t = e / d, k = e - t * d;
            c128 acc = U[e] + b2[k];
            for (int m = 0; m < h; ++m) cmac(acc, W2[(long long)k * h + m], AZ[t * h + m]);
            H[e] = acc;
            if (sv) sv[2 * T * d + T * h + e] = acc;
        }
        __syncthreads();
    }
    const c128* wO = th + enc_base(md, md.L);
    double re = 0.0, im = 0.0;
    for (int e = threadIdx.x; e < T * d; e += blockDim.x) {
        const c128 v = clncosh(H[e]), w = wO[e % d];
        re += w.re * v.re - w.im * v.im;
        im += w.re * v.im + w.im * v.re;
    }
    re = block_sum(re, sh);
    im = block_sum(im, sh);
    const c128 bO = wO[d];
    return mk<double>(re + bO.re, im + bO.im);
}

__global__ void __launch_bounds__(VT) vit_forward_kernel(ModelDesc md, const c128* __restrict__ th,
                                                         const int8_t* __restrict__ x, long long ns,
                                                         c128* __restrict__ Z, c128* __restrict__ logpsi) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = md.vT, d = md.vd, h = md.vh, N = md.N;
    c128* H = reinterpret_cast<c128*>(smem);
    c128* V = H + T * d;
    c128* U = V + T * d;
    c128* AZ = U + T * d;
    float* xs = reinterpret_cast<float*>(AZ + T * h);
    __shared__ double sh[32];
    for (long long s = blockIdx.x; s < ns; s += gridDim.x) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) xs[i] = (float)x[s * N + i];
        __syncthreads();
        const c128 lp = vit_forward_cta(md, th, xs, H, V, U, AZ, Z ? Z + s * md.vsave : nullptr, sh);
        if (threadIdx.x == 0) logpsi[s] = lp;
        __syncthreads();
    }
}

// column s of O (parameter-major); zero for padding columns n_s <= s < ldo
__global__ void __launch_bounds__(VT) vit_jacobian_kernel(ModelDesc md, const c128* __restrict__ th,
                                                          const c128* __restrict__ Z, const int8_t* __restrict__ x,
                                                          long long ns, c128* __restrict__ O, long long ldo) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = md.vT, p = md.vp, d = md.vd, h = md.vh, N = md.N, L = md.L;
    c128* GH = reinterpret_cast<c128*>(smem);
    c128* GU = GH + T * d;
    c128* GV = GU + T * d;
    c128* GZ = GV + T * d;
    c128* AZ = GZ + T * h;
    float* xs = reinterpret_cast<float*>(AZ + T * h);
    const c128 zero = mk<double>(0.0, 0.0);
    for (long long s = blockIdx.x; s < ldo; s += gridDim.x) {
        if (s >= ns) {
            for (long long k = threadIdx.x; k < md.n_p; k += blockDim.x) O[k * ldo + s] = zero;
            continue;
        }
        for (int i = threadIdx.x; i < N; i += blockDim.x) xs[i] = (float)x[s * N + i];
        const c128* sv = Z + s * md.vsave;
        const c128* HL = L > 0 ? sv + h_out(md, L - 1) : sv;
        const long long ob = enc_base(md, L);
        const c128* wO = th + ob;
        // output layer: O(w_O)_k = sum_t lncosh(h_tk), O(b_O) = 1; g_h = w_O tanh(h)
        for (int k = threadIdx.x; k < d; k += blockDim.x) {
            c128 acc = zero;
            for (int t = 0; t < T; ++t) acc = acc + clncosh(HL[t * d + k]);
            O[(ob + k) * ldo + s] = acc;
        }
        if (threadIdx.x == 0) O[(ob + d) * ldo + s] = mk<double>(1.0, 0.0);
        for (int e = threadIdx.x; e < T * d; e += blockDim.x) GH[e] = wO[e % d] * ctanh(HL[e]);
        __syncthreads();
        for (int l = L - 1; l >= 0; --l) {
            const long long po = enc_base(md, l);
            const c128* A = th + po;
            const c128* WV = A + (long long)T * T;
            const c128* W1 = WV + (long long)d * d;
            const c128* W2 = W1 + (long long)h * d + h;
            const c128* v = sv + lay_base(md, l);
            const c128* u = v + T * d;
            const c128* z = u + T * d;
            const c128* hin = l > 0 ? sv + h_out(md, l - 1) : sv;
            const long long oA = po, oWV = oA + (long long)T * T, oW1 = oWV + (long long)d * d,
                            ob1 = oW1 + (long long)h * d, oW2 = ob1 + h, ob2 = oW2 + (long long)d * h;
            for (int e = threadIdx.x; e < T * h; e += blockDim.x) {  // g_z = (W_2^T g_h) tanh(z); a = lncosh z
                const int t = e / h, m = e - t * h;
                c128 acc = zero;
                for (int k = 0; k < d; ++k) cmac(acc, W2[(long long)k * h + m], GH[t * d + k]);
                GZ[e] = acc * ctanh(z[e]);
                AZ[e] = clncosh(z[e]);
            }
            __syncthreads();
            for (int q = threadIdx.x; q < d * h; q += blockDim.x) {  // O(W_2)[k][m] = sum_t g_h[t][k] a[t][m]
                const int k = q / h, m = q - k * h;
                c128 acc = zero;
                for (int t = 0; t < T; ++t) cmac(acc, GH[t * d + k], AZ[t * h + m]);
                O[(oW2 + q) * ldo + s] = acc;
            }
            for (int k = threadIdx.x; k < d; k += blockDim.x) {  // O(b_2) = sum_t g_h[t]
                c128 acc = zero;
                for (int t = 0; t < T; ++t) acc = acc + GH[t * d + k];
                O[(ob2 + k) * ldo + s] = acc;
            }
            for (int q = threadIdx.x; q < h * d; q += blockDim.x) {  // O(W_1)[m][j] = sum_t g_z[t][m] u[t][j]
                const int m = q / d, j = q - m * d;
                c128 acc = zero;
                for (int t = 0; t < T; ++t) cmac(acc, GZ[t * h + m], u[t * d + j]);
                O[(oW1 + q) * ldo + s] = acc;
            }
            for (int m = threadIdx.x; m < h; m += blockDim.x) {  // O(b_1) = sum_t g_z[t]
                c128 acc = zero;
                for (int t = 0; t < T; ++t) acc = acc + GZ[t * h + m];
                O[(ob1 + m) * ldo + s] = acc;
            }
            for (int e = threadIdx.x; e < T * d; e += blockDim.x) {  // g_u = g_h + W_1^T g_z
                const int t = e / d, j = e - t * d;
                c128 acc = GH[e];
                for (int m = 0; m < h; ++m) cmac(acc, W1[(long long)m * d + j], GZ[t * h + m]);
                GU[e] = acc;
            }
            __syncthreads();
            for (int q = threadIdx.x; q < T * T; q += blockDim.x) {  // O(A)[t][r] = sum_k g_u[t][k] v[r][k]
                const int t = q / T, r = q - t * T;
                c128 acc = zero;
                for (int k = 0; k < d; ++k) cmac(acc, GU[t * d + k], v[r * d + k]);
                O[(oA + q) * ldo + s] = acc;
            }
            for (int e = threadIdx.x; e < T * d; e += blockDim.x) {  // g_v[r] = sum_t A[t][r] g_u[t]
                const int r = e / d, k = e - r * d;
                c128 acc = zero;
                for (int t = 0; t < T; ++t) cmac(acc, A[(long long)t * T + r], GU[t * d + k]);
                GV[e] = acc;
            }
            __syncthreads();
            for (int q = threadIdx.x; q < d * d; q += blockDim.x) {  // O(W_V)[k][j] = sum_r g_v[r][k] h[r][j]
                const int k = q / d, j = q - k * d;
                c128 acc = zero;
                for (int r = 0; r < T; ++r) cmac(acc, GV[r * d + k], hin[r * d + j]);
                O[(oWV + q) * ldo + s] = acc;
            }
            for (int e = threadIdx.x; e < T * d; e += blockDim.x) {  // g_h = g_u + W_V^T g_v
                const int r = e / d, j = e - r * d;
                c128 acc = GU[e];
                for (int k = 0; k < d; ++k) cmac(acc, WV[(long long)k * d + j], GV[r * d + k]);
                GH[e] = acc;
            }
            __syncthreads();
        }
        for (int q = threadIdx.x; q < d * p; q += blockDim.x) {  // O(W_E)[k][j] = sum_t g_h[t][k] x[t p + j]
            const int k = q / p, j = q - k * p;
            c128 acc = zero;
            for (int t = 0; t < T; ++t) {
                const double xv = xs[t * p + j];
                acc.re = fma(GH[t * d + k].re, xv, acc.re);
                acc.im = fma(GH[t * d + k].im, xv, acc.im);
            }
            O[(long long)q * ldo + s] = acc;
        }
        for (int k = threadIdx.x; k < d; k += blockDim.x) {  // O(b_E) = sum_t g_h[t]
            c128 acc = zero;
            for (int t = 0; t < T; ++t) acc = acc + GH[t * d + k];
            O[((long long)d * p + k) * ldo + s] = acc;
        }
        __syncthreads();
    }
}

// E_loc terms 2 c J_b sign psi(x^{ij}) / psi(x): a full forward of each connected configuration
__global__ void __launch_bounds__(VT) vit_conn_kernel(ModelDesc md, const c128* __restrict__ th,
                                                      const c128* __restrict__ logpsi, const int8_t* __restrict__ x,
                                                      HamDesc hd, const int32_t* __restrict__ cbond,
                                                      const int32_t* __restrict__ csamp,
                                                      const long long* __restrict__ nconn_ptr,
                                                      c128* __restrict__ terms) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = md.vT, d = md.vd, h = md.vh, N = md.N;
    c128* H = reinterpret_cast<c128*>(smem);
    c128* V = H + T * d;
    c128* U = V + T * d;
    c128* AZ = U + T * d;
    float* xs = reinterpret_cast<float*>(AZ + T * h);
    __shared__ double sh[32];
    const long long nconn = *nconn_ptr;
    for (long long c = blockIdx.x; c < nconn; c += gridDim.x) {
        const long long s = csamp[c];
        const int b = cbond[c];
        const int bi = hd.bond_ij[2 * b], bj = hd.bond_ij[2 * b + 1];
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const float v = (float)x[s * N + i];
            xs[i] = (i == bi || i == bj) ? -v : v;
        }
        __syncthreads();
        const c128 lp = vit_forward_cta(md, th, xs, H, V, U, AZ, nullptr, sh);
        if (threadIdx.x == 0) {
            const c128 dl = lp - logpsi[s];
            const double m = exp(dl.re);
            double sn, cs;
            sincos(dl.im, &sn, &cs);
            const double f = 2.0 * hd.c * hd.bond_J[b] * (double)hd.sign_rule;
            terms[c] = mk<double>(f * m * cs, f * m * sn);
        }
        __syncthreads();
    }
}

size_t fwd_smem(const ModelDesc& md) {
    return (3ull * md.vT * md.vd + (size_t)md.vT * md.vh) * sizeof(c128) + (size_t)md.N * sizeof(float);
}
size_t jac_smem(const ModelDesc& md) {
    return (3ull * md.vT * md.vd + 2ull * md.vT * md.vh) * sizeof(c128) + (size_t)md.N * sizeof(float);
}
unsigned grid_of(long long n) { return (unsigned)(n < 1 ? 1 : (n > 16384 ? 16384 : n)); }

}  // namespace

cudaError_t launch_vit_forward(const ModelDesc& md, const c128* th, const int8_t* x, long long ns, c128* Z,
                               c128* logpsi, cudaStream_t st) {
    if (ns <= 0) return cudaSuccess;
    const size_t sm = fwd_smem(md);
    cudaError_t e = cudaFuncSetAttribute(vit_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    count_launch();
    vit_forward_kernel<<<grid_of(ns), VT, sm, st>>>(md, th, x, ns, Z, logpsi);
    return cudaGetLastError();
}

cudaError_t launch_vit_jacobian(const ModelDesc& md, const c128* th, const c128* Z, const int8_t* x, long long ns,
                                c128* O, long long ldo, cudaStream_t st) {
    if (ldo <= 0) return cudaSuccess;
    const size_t sm = jac_smem(md);
    cudaError_t e = cudaFuncSetAttribute(vit_jacobian_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    count_launch();
    vit_jacobian_kernel<<<grid_of(ldo), VT, sm, st>>>(md, th, Z, x, ns, O, ldo);
    return cudaGetLastError();
}

cudaError_t launch_vit_conn_terms(const ModelDesc& md, const c128* th, const c128* logpsi, const int8_t* x,
                                  const HamDesc& h, const int32_t* conn_bond, const int32_t* conn_sample,
                                  const long long* nconn_ptr, long long max_conn, c128* terms, cudaStream_t st) {
    if (max_conn <= 0) return cudaSuccess;
    const size_t sm = fwd_smem(md);
    cudaError_t e = cudaFuncSetAttribute(vit_conn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    count_launch();
    vit_conn_kernel<<<grid_of(max_conn), VT, sm, st>>>(md, th, logpsi, x, h, conn_bond, conn_sample, nconn_ptr,
                                                       terms);
    return cudaGetLastError();
}

}  // namespace nqs
