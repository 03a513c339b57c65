// Complex NQS forward pass, per-sample backward pass and parameter-major Jacobian
// (Sec. 2: O_k(x) = d ln psi(x) / d theta_k, holomorphic; RBM and ln cosh FFNN).
//
// Layouts: activations Z_l and backward signals G_l are sample-major [n_s][width];
// the Jacobian is parameter-major O[k * ldo + s] so that every later stage
// (centring, force, Gram) streams contiguous sample rows.
#include "internal.cuh"

namespace nqs {

static int build_vit_desc(const nqs_model* m, long long ns, ModelDesc* md) {
    const int N = m->widths[0], p = m->widths[1], d = m->widths[2], h = m->widths[3], L = m->n_layers;
    if (N < 2 || N > MAXN || p < 1 || N % p || d < 1 || d > 128 || h < 1 || h > 256 || L < 0 || L > MAXL)
        return NQS_ERR_INVALID_ARG;
    const int T = N / p;
    if (T > 64 || (long long)T * (3 * d + h) > VIT_SMEM_CX) return NQS_ERR_INVALID_ARG;
    md->kind = NQS_VIT;
    md->L = L;
    md->N = N;
    for (int i = 0; i < 4; ++i) md->widths[i] = m->widths[i];
    md->maxw = d > h ? d : h;
    md->vp = p;
    md->vT = T;
    md->vd = d;
    md->vh = h;
    md->vE = (long long)T * T + (long long)d * d + 2LL * h * d + h + d;
    md->vsave = (long long)T * d + (long long)L * (3LL * T * d + (long long)T * h);
    const long long np = (long long)d * p + d + L * md->vE + d + 1;
    if (np > 0x7fffffffLL) return NQS_ERR_INVALID_ARG;
    md->n_p = (int)np;
    (void)ns;
    return NQS_OK;
}

int build_model_desc(const nqs_model* m, long long ns, ModelDesc* md) {
    if (m && m->kind == NQS_VIT && m->widths) {
        *md = ModelDesc{};
        return build_vit_desc(m, ns, md);
    }
    if (!m || !m->widths || m->n_layers < 1 || m->n_layers > MAXL) return NQS_ERR_INVALID_ARG;
    *md = ModelDesc{};
    md->kind = m->kind;
    md->L = m->n_layers;
    for (int i = 0; i <= m->n_layers; ++i) {
        if (m->widths[i] < 1 || m->widths[i] > MAXW) return NQS_ERR_INVALID_ARG;
        md->widths[i] = m->widths[i];
    }
    md->N = m->widths[0];
    if (md->N > MAXN) return NQS_ERR_INVALID_ARG;
    md->maxw = 0;
    for (int i = 0; i <= md->L; ++i) md->maxw = md->widths[i] > md->maxw ? md->widths[i] : md->maxw;
    long long wt = 0, z = 0;
    if (m->kind == NQS_RBM) {
        if (m->n_layers != 1) return NQS_ERR_INVALID_ARG;
        const int N = md->widths[0], M = md->widths[1];
        md->aoff = 0;
        md->boff[0] = N;
        md->woff[0] = N + M;
        md->n_p = N + M + M * N;
        md->wtoff[0] = 0;
        md->zoff[0] = 0;
    } else if (m->kind == NQS_FFNN) {
        if (md->widths[md->L] != 1) return NQS_ERR_INVALID_ARG;
        long long p = 0;
        for (int l = 0; l < md->L; ++l) {
            const long long o = md->widths[l + 1], in = md->widths[l];
            md->woff[l] = p;
            md->boff[l] = p + o * in;
            p += o * in + o;
            md->wtoff[l] = wt;
            wt += o * in;
            md->zoff[l] = z;
            z += ns * o;
        }
        md->n_p = (int)p;
    } else {
        return NQS_ERR_INVALID_ARG;
    }
    return NQS_OK;
}

long long model_wt_elems(const ModelDesc& md) {
    if (md.kind == NQS_VIT) return 0;
    long long t = 0;
    for (int l = 0; l < md.L; ++l) t += (long long)md.widths[l + 1] * md.widths[l];
    return t;
}
long long model_z_elems(const ModelDesc& md, long long ns) {
    if (md.kind == NQS_VIT) return ns * md.vsave;
    long long t = 0;
    for (int l = 0; l < md.L; ++l) t += ns * md.widths[l + 1];
    return t;
}

// ------------------------------------------------------------------ parameters
template <typename R>
__global__ void prepare_params_kernel(ModelDesc md, const c128* __restrict__ th, cx<R>* __restrict__ thR,
                                      cx<R>* __restrict__ wt) {
    const long long n = md.n_p;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const cx<R> v = ccast<R>(th[p]);
        thR[p] = v;
        for (int l = 0; l < (md.kind == NQS_VIT ? 0 : md.L); ++l) {
            const long long o = md.widths[l + 1], in = md.widths[l];
            if (p >= md.woff[l] && p < md.woff[l] + o * in) {
                const long long q = p - md.woff[l];
                const long long j = q / in, k = q % in;
                wt[md.wtoff[l] + k * o + j] = v;
            }
        }
    }
}

// ------------------------------------------------------------------ forward
// One CTA evaluates TR samples through every layer with activations in shared
// memory; weights are read transposed (W^T: [in][out]) so that consecutive
// threads (consecutive output units) read consecutive addresses.
template <typename R>
__global__ void __launch_bounds__(256) fwd_kernel(ModelDesc md, const cx<R>* __restrict__ th,
                                                   const cx<R>* __restrict__ wt,
                                                   const int8_t* __restrict__ x, long long ns, int TR,
                                                   cx<R>* __restrict__ Z, c128* __restrict__ logpsi) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* A = reinterpret_cast<cx<R>*>(smem_raw);
    const int ld = md.maxw;
    cx<R>* B = A + (size_t)TR * ld;
    const long long s0 = (long long)blockIdx.x * TR;
    const int rows = (int)((ns - s0) < TR ? (ns - s0) : TR);
    const int N = md.N;
    for (int idx = threadIdx.x; idx < TR * N; idx += blockDim.x) {
        const int r = idx / N, k = idx % N;
        const R v = (r < rows) ? (R)x[(s0 + r) * N + k] : R(0);
        A[r * ld + k] = mk<R>(v, R(0));
    }
    __syncthreads();
    for (int l = 0; l < md.L; ++l) {
        const int out = md.widths[l + 1], in = md.widths[l];
        const cx<R>* W = wt + md.wtoff[l];
        const cx<R>* bias = th + md.boff[l];
        const int groups = (TR / 4) * out;
        const bool last_ffnn = (md.kind == NQS_FFNN) && (l == md.L - 1);
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
                if (r < rows) {
                    if (last_ffnn) {
                        logpsi[s0 + r] = ccast<double>(acc[q]);
                    } else {
                        Z[md.zoff[l] + (s0 + r) * out + j] = acc[q];
                        B[r * ld + j] = clncosh(acc[q]);
                    }
                } else {
                    B[r * ld + j] = mk<R>(R(0), R(0));
                }
            }
        }
        __syncthreads();
        cx<R>* t = A;
        A = B;
        B = t;
    }
    if (md.kind == NQS_RBM) {
        // ln psi = a.x + sum_j lncosh(z_j): A holds lncosh(z), B still holds x.
        const int M = md.widths[1];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int r = wid; r < rows; r += nw) {
            cx<R> acc = mk<R>(R(0), R(0));
            for (int j = lane; j < M; j += 32) acc = acc + A[r * ld + j];
            for (int i = lane; i < N; i += 32) cmac(acc, th[md.aoff + i], B[r * ld + i]);
            acc = warp_sum(acc);
            if (lane == 0) logpsi[s0 + r] = ccast<double>(acc);
        }
    }
}

// ------------------------------------------------------------------ backward
// g_h(L-1) = W_L (one output); for hidden layers l = L-2..0:
//   g_z = g_h * tanh(z_l)   (stored as G_l),   g_h(l-1) = W_l^T g_z.
template <typename R>
__global__ void __launch_bounds__(256) bwd_kernel(ModelDesc md, const cx<R>* __restrict__ th,
                                                   const cx<R>* __restrict__ Z, long long ns, int TR,
                                                   cx<R>* __restrict__ G) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* GH = reinterpret_cast<cx<R>*>(smem_raw);
    const int ld = md.maxw;
    cx<R>* GZ = GH + (size_t)TR * ld;
    const long long s0 = (long long)blockIdx.x * TR;
    const int rows = (int)((ns - s0) < TR ? (ns - s0) : TR);
    const int L = md.L;
    {
        const int w = md.widths[L - 1];
        const cx<R>* WL = th + md.woff[L - 1];
        for (int idx = threadIdx.x; idx < TR * w; idx += blockDim.x) {
            const int r = idx / w, k = idx % w;
            GH[r * ld + k] = WL[k];
        }
    }
    __syncthreads();
    for (int l = L - 2; l >= 0; --l) {
        const int out = md.widths[l + 1], in = md.widths[l];
        for (int idx = threadIdx.x; idx < TR * out; idx += blockDim.x) {
            const int r = idx / out, j = idx % out;
            cx<R> gz = mk<R>(R(0), R(0));
            if (r < rows) {
                const long long zi = md.zoff[l] + (s0 + r) * out + j;
                gz = GH[r * ld + j] * ctanh(Z[zi]);
                G[zi] = gz;
            }
            GZ[r * ld + j] = gz;
        }
        __syncthreads();
        if (l > 0) {
            const cx<R>* W = th + md.woff[l];  // [out][in]
            const int groups = (TR / 4) * in;
            for (int g = threadIdx.x; g < groups; g += blockDim.x) {
                const int rg = g / in, k = g % in;
                cx<R> acc[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = mk<R>(R(0), R(0));
                for (int j = 0; j < out; ++j) {
                    const cx<R> w = W[(long long)j * in + k];
#pragma unroll
                    for (int q = 0; q < 4; ++q) cmac(acc[q], GZ[(4 * rg + q) * ld + j], w);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) GH[(4 * rg + q) * ld + k] = acc[q];
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------ Jacobian
// Layer l: O(W_l[j][k]) = g_z[j] h_{l-1}[k], O(b_l[j]) = g_z[j]
// (FFNN output layer: g_z = 1; RBM: g_z = tanh(z), h = x, plus O(a_i) = x_i).
// One CTA: 32 samples (one per lane) x JC output units x KC inputs; every warp
// store writes 32 consecutive samples of one parameter row.
constexpr int JAC_TS = 32;
constexpr int JAC_JC = 64;  // output units per CTA: every h_{l-1} value is computed once per tile
constexpr int JAC_KC = 32;
template <typename R>
__global__ void __launch_bounds__(256) jac_kernel(ModelDesc md, int l, const cx<R>* __restrict__ Z,
                                                   const cx<R>* __restrict__ G,
                                                   const int8_t* __restrict__ x, long long ns,
                                                   cx<R>* __restrict__ O, long long ldo) {
    __shared__ cx<R> HT[JAC_KC][JAC_TS + 1];
    __shared__ cx<R> GT[JAC_JC][JAC_TS + 1];
    const int out = md.widths[l + 1], in = md.widths[l];
    const long long s0 = (long long)blockIdx.x * JAC_TS;
    const int j0 = blockIdx.y * JAC_JC;
    const int jn = (out - j0) < JAC_JC ? (out - j0) : JAC_JC;
    const int k0 = blockIdx.z * JAC_KC;
    const int kn = (in - k0) < JAC_KC ? (in - k0) : JAC_KC;
    const bool rbm = md.kind == NQS_RBM;
    const bool outl = (!rbm) && (l == md.L - 1);
    for (int idx = threadIdx.x; idx < JAC_TS * kn; idx += blockDim.x) {
        const int r = idx / kn, kk = idx % kn;
        const long long s = s0 + r;
        cx<R> h = mk<R>(R(0), R(0));
        if (s < ns) {
            if (l == 0) h = mk<R>((R)x[s * md.N + k0 + kk], R(0));
            else h = clncosh(Z[md.zoff[l - 1] + s * in + k0 + kk]);
        }
        HT[kk][r] = h;
    }
    for (int idx = threadIdx.x; idx < JAC_TS * jn; idx += blockDim.x) {
        const int r = idx / jn, jj = idx % jn;
        const long long s = s0 + r;
        cx<R> g = mk<R>(R(0), R(0));
        if (s < ns) {
            if (outl) g = mk<R>(R(1), R(0));
            else if (rbm) g = ctanh(Z[md.zoff[0] + s * out + j0 + jj]);
            else g = G[md.zoff[l] + s * out + j0 + jj];
        }
        GT[jj][r] = g;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long s = s0 + lane;
    if (s >= ldo) return;
    const bool live = s < ns;
    const cx<R> zero = mk<R>(R(0), R(0));
    // warp w writes rows (j0 + jj, k0 .. k0 + kn) for jj = w, w + nw, ...: 32 samples (one
    // 512-byte segment for c128) per store, four independent stores in flight per step
    for (int jj = wid; jj < jn; jj += nw) {
        const cx<R> g = live ? GT[jj][lane] : zero;
        cx<R>* orow = O + (md.woff[l] + (long long)(j0 + jj) * in + k0) * ldo + s;
        int kk = 0;
        for (; kk + 4 <= kn; kk += 4) {
            const cx<R> v0 = g * HT[kk][lane], v1 = g * HT[kk + 1][lane];
            const cx<R> v2 = g * HT[kk + 2][lane], v3 = g * HT[kk + 3][lane];
            orow[(long long)kk * ldo] = v0;
            orow[(long long)(kk + 1) * ldo] = v1;
            orow[(long long)(kk + 2) * ldo] = v2;
            orow[(long long)(kk + 3) * ldo] = v3;
        }
        for (; kk < kn; ++kk) orow[(long long)kk * ldo] = g * HT[kk][lane];
    }
    if (blockIdx.z == 0) {
        for (int jj = wid; jj < jn; jj += nw)
            O[(md.boff[l] + j0 + jj) * ldo + s] = live ? GT[jj][lane] : zero;
    }
    if (rbm && blockIdx.y == 0) {
        for (int kk = wid; kk < kn; kk += nw)
            O[(md.aoff + k0 + kk) * ldo + s] = live ? HT[kk][lane] : zero;
    }
}

// ------------------------------------------------------------------ launchers
static int pick_tr(int maxw, size_t csize) {
    // two activation buffers of TR x maxw complex values within ~192 KB
    long long tr = 196608LL / (2LL * maxw * (long long)csize);
    tr = tr > 32 ? 32 : tr;
    tr = (tr / 4) * 4;
    return tr < 4 ? 4 : (int)tr;
}

template <typename R>
static cudaError_t forward_t(const ModelDesc& md, const void* thR, const void* wtR, const int8_t* x,
                             long long ns, void* Z, c128* logpsi, cudaStream_t st) {
    if (ns <= 0) return cudaSuccess;
    const int TR = pick_tr(md.maxw, sizeof(cx<R>));
    const size_t smem = 2ull * TR * md.maxw * sizeof(cx<R>);
    cudaError_t e = cudaFuncSetAttribute(fwd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)((ns + TR - 1) / TR);
    count_launch();
    fwd_kernel<R><<<grid, 256, smem, st>>>(md, (const cx<R>*)thR, (const cx<R>*)wtR, x, ns, TR,
                                           (cx<R>*)Z, logpsi);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t backward_t(const ModelDesc& md, const void* thR, const void* Z, long long ns,
                              void* G, cudaStream_t st) {
    if (md.kind != NQS_FFNN || md.L < 2 || ns <= 0) return cudaSuccess;
    const int TR = pick_tr(md.maxw, sizeof(cx<R>));
    const size_t smem = 2ull * TR * md.maxw * sizeof(cx<R>);
    cudaError_t e = cudaFuncSetAttribute(bwd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)((ns + TR - 1) / TR);
    count_launch();
    bwd_kernel<R><<<grid, 256, smem, st>>>(md, (const cx<R>*)thR, (const cx<R>*)Z, ns, TR, (cx<R>*)G);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t jac_t(const ModelDesc& md, const void* Z, const void* G, const int8_t* x,
                         long long ns, void* O, long long ldo, cudaStream_t st) {
    if (ldo <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < md.L; ++l) {
        const int out = md.widths[l + 1], in = md.widths[l];
        dim3 grid((unsigned)((ldo + JAC_TS - 1) / JAC_TS), (unsigned)((out + JAC_JC - 1) / JAC_JC),
                  (unsigned)((in + JAC_KC - 1) / JAC_KC));
        count_launch();
        jac_kernel<R><<<grid, 256, 0, st>>>(md, l, (const cx<R>*)Z, (const cx<R>*)G, x, ns, (cx<R>*)O, ldo);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_prepare_params(int prec, const ModelDesc& md, const void* theta, void* thR,
                                  void* wtR, cudaStream_t st) {
    const int grid = (md.n_p + 255) / 256 < 4096 ? (md.n_p + 255) / 256 : 4096;
    if (prec == NQS_FP64) {
        count_launch();
        prepare_params_kernel<double><<<grid, 256, 0, st>>>(md, (const c128*)theta, (c128*)thR, (c128*)wtR);
    } else {
        count_launch();
        prepare_params_kernel<float><<<grid, 256, 0, st>>>(md, (const c128*)theta, (c64*)thR, (c64*)wtR);
    }
    return cudaGetLastError();
}
cudaError_t launch_forward(int prec, const ModelDesc& md, const void* thR, const void* wtR,
                           const int8_t* x, long long ns, void* Z, c128* logpsi, cudaStream_t st) {
    if (md.kind == NQS_VIT)
        return prec == NQS_FP64 ? launch_vit_forward(md, (const c128*)thR, x, ns, (c128*)Z, logpsi, st)
                                : cudaErrorNotSupported;
    return prec == NQS_FP64 ? forward_t<double>(md, thR, wtR, x, ns, Z, logpsi, st)
                            : forward_t<float>(md, thR, wtR, x, ns, Z, logpsi, st);
}
cudaError_t launch_backward(int prec, const ModelDesc& md, const void* thR, const void* Z,
                            long long ns, void* G, cudaStream_t st) {
    if (md.kind == NQS_VIT) return cudaSuccess;  // the transformer's backward runs in launch_jac_write
    return prec == NQS_FP64 ? backward_t<double>(md, thR, Z, ns, G, st)
                            : backward_t<float>(md, thR, Z, ns, G, st);
}
cudaError_t launch_jac_write(int prec, const ModelDesc& md, const void* thR, const void* Z, const void* G,
                             const int8_t* x, long long ns, void* O, long long ldo, cudaStream_t st) {
    if (md.kind == NQS_VIT)
        return prec == NQS_FP64 ? launch_vit_jacobian(md, (const c128*)thR, (const c128*)Z, x, ns, (c128*)O, ldo, st)
                                : cudaErrorNotSupported;
    return prec == NQS_FP64 ? jac_t<double>(md, Z, G, x, ns, O, ldo, st)
                            : jac_t<float>(md, Z, G, x, ns, O, ldo, st);
}

}  // namespace nqs
