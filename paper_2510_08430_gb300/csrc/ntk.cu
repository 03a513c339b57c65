// Sample-space (NTK) solve, the comparator of the block-layer step (Sec. 2: the full-QGT
// update written in sample space; equal to it by the push-through identity when no
// eigenvalue is cut):
//   dtheta = -eta X^H (X X^H + lambda I)^{-1} eps,   X = dO / sqrt(N),  eps = e / sqrt(N).
// The N_s x N_s Gram is formed by the parameter-space Gram kernels on the transposed
// (sample-major) dO: they give S_T[s][t] = sum_k conj(dO_k(s)) dO_k(t) / N = conj((X X^H)[s][t]),
// so (S_T + lambda I) u = conj(eps) is solved and z = conj(u).
#include "internal.cuh"

namespace nqs {

// Y[s][k] = (R) dO[k][s] through 32 x 32 shared-memory tiles.
template <typename R>
__global__ void __launch_bounds__(256) transpose_kernel(const c128* __restrict__ O, long long ldo, long long ns,
                                                         long long np, cx<R>* __restrict__ Y, long long ldy) {
    __shared__ c128 t[32][33];
    const long long s0 = (long long)blockIdx.x * 32, k0 = (long long)blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const long long k = k0 + r, s = s0 + tx;
        t[r][tx] = (k < np && s < ns) ? O[k * ldo + s] : mk<double>(0.0, 0.0);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const long long s = s0 + r, k = k0 + tx;
        if (s < ns && k < ldy) Y[s * ldy + k] = ccast<R>(t[tx][r]);
    }
}

// rhs[s] = conj(e[s]) / sqrt(N)
__global__ void ntk_rhs_kernel(const c128* __restrict__ e, long long ns, c128* __restrict__ rhs) {
    const double f = 1.0 / sqrt((double)ns);
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < ns; s += (long long)gridDim.x * blockDim.x)
        rhs[s] = f * cconj(e[s]);
}

// dtheta[k] = -eta / sqrt(N) conj(sum_s dO[k][s] u[s])
__global__ void __launch_bounds__(256) ntk_back_kernel(const c128* __restrict__ O, long long ldo, long long ns,
                                                        const c128* __restrict__ u, double eta,
                                                        c128* __restrict__ dtheta) {
    __shared__ double sh[32];
    const c128* row = O + blockIdx.x * ldo;
    c128 acc = mk<double>(0.0, 0.0);
    for (long long s = threadIdx.x; s < ns; s += blockDim.x) cmac(acc, row[s], u[s]);
    acc.re = block_sum(acc.re, sh);
    acc.im = block_sum(acc.im, sh);
    if (threadIdx.x == 0) dtheta[blockIdx.x] = (-eta / sqrt((double)ns)) * cconj(acc);
}

cudaError_t launch_ntk_transpose(int prec, const c128* O, long long ldo, long long ns, long long np, void* Y,
                                 long long ldy, cudaStream_t st) {
    const dim3 grid((unsigned)((ns + 31) / 32), (unsigned)((ldy + 31) / 32));
    count_launch();
    if (prec == NQS_FP32)
        transpose_kernel<float><<<grid, 256, 0, st>>>(O, ldo, ns, np, (c64*)Y, ldy);
    else
        transpose_kernel<double><<<grid, 256, 0, st>>>(O, ldo, ns, np, (c128*)Y, ldy);
    return cudaGetLastError();
}

cudaError_t launch_ntk_rhs(const c128* e, long long ns, c128* rhs, cudaStream_t st) {
    count_launch();
    ntk_rhs_kernel<<<(unsigned)((ns + 255) / 256 < 1024 ? (ns + 255) / 256 : 1024), 256, 0, st>>>(e, ns, rhs);
    return cudaGetLastError();
}

cudaError_t launch_ntk_back(const c128* O, long long ldo, long long ns, long long np, const c128* u, double eta,
                            c128* dtheta, cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    count_launch();
    ntk_back_kernel<<<(unsigned)np, 256, 0, st>>>(O, ldo, ns, u, eta, dtheta);
    return cudaGetLastError();
}

}  // namespace nqs
