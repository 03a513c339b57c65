// Inverse-metric diagnostics of the block-layer QGT (Eq. 4, Sec. 3): with A and B the
// pseudo-inverses of two shifted QGTs,
//   (a) F(A, B)     = Tr[A^H B] / (|A|_F |B|_F),
//   (b) eps_F(A, B) = |A - B|_F / |B|_F,
//   (c) kappa(A)    = lambda_max(A) / lambda_min(A)   (over the eigenvalues the cutoff keeps),
//   (d) r_lambda    = Pearson correlation of the two spectra, each sorted in descending order.
// From the eigen-decompositions S~_a = U_a diag(s_a) U_a^H and S~_b = U_b diag(s_b) U_b^H,
// A = U_a diag(a) U_a^H with a_i = keep_i / s_a,i (and b likewise):
//   Tr[A^H B] = sum_ij a_i b_j |(U_a^H U_b)_ij|^2,  |A|_F^2 = sum_i a_i^2,
//   |A - B|_F^2 = |A|_F^2 + |B|_F^2 - 2 Tr[A^H B].
// Also: Born weights |psi|^2 / Z of an enumerated Hilbert space (the exact QGT's sample
// weights), and the restriction of a full QGT to its diagonal blocks.
#include "internal.cuh"

namespace nqs {
namespace {

constexpr int DT = 32;  // tile edge of the overlap kernel

// w_s = exp(2 Re ln psi_s - m) / sum_t exp(2 Re ln psi_t - m), m = max_t 2 Re ln psi_t (one CTA)
__global__ void __launch_bounds__(1024) born_weights_kernel(const c128* __restrict__ lp, long long n,
                                                            double* __restrict__ w) {
    __shared__ double sh[32];
    __shared__ double smax;
    double m = -1e300;
    for (long long s = threadIdx.x; s < n; s += blockDim.x) m = fmax(m, 2.0 * lp[s].re);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = -1e300;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) mm = fmax(mm, sh[k]);
        smax = mm;
    }
    __syncthreads();
    const double mx = smax;
    double z = 0.0;
    for (long long s = threadIdx.x; s < n; s += blockDim.x) z += exp(2.0 * lp[s].re - mx);
    z = block_sum(z, sh);
    for (long long s = threadIdx.x; s < n; s += blockDim.x) w[s] = exp(2.0 * lp[s].re - mx) / z;
}

// out = S with every entry outside the diagonal blocks set to zero (lower triangle; n x n)
__global__ void block_restrict_kernel(const c128* __restrict__ S, long long n, const long long* __restrict__ blk_of,
                                      c128* __restrict__ out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / n, c = e % n;
        out[e] = (blk_of[r] == blk_of[c]) ? S[e] : mk<double>(0.0, 0.0);
    }
}

struct OffTab {
    int64_t v[MAXB + 1];
};

__global__ void block_index_kernel(const OffTab off, int nb, long long* __restrict__ blk_of) {
    const int b = blockIdx.x;
    if (b >= nb) return;
    for (long long k = off.v[b] + threadIdx.x; k < off.v[b + 1]; k += blockDim.x) blk_of[k] = b;
}

__device__ __forceinline__ double keep_inv(double s, double thr) { return s > thr ? 1.0 / s : 0.0; }

// Thresholds of the two spectra (one CTA): thr = cutoff * max(s) (mode 0) or cutoff.
__global__ void thresholds_kernel(const double* __restrict__ ev_a, const double* __restrict__ ev_b, long long n,
                                  double cutoff, int mode, double* __restrict__ thr) {
    if (threadIdx.x == 0) {
        thr[0] = mode == 0 ? cutoff * ev_a[n - 1] : cutoff;  // ev ascending
        thr[1] = mode == 0 ? cutoff * ev_b[n - 1] : cutoff;
    }
}

// partial[tile] = sum over the 32 x 32 tile (i, j) of a_i b_j |sum_r conj(Ua[i][r]) Ub[j][r]|^2
__global__ void __launch_bounds__(256) overlap_kernel(long long n, const double* __restrict__ sig_a,
                                                      const c128* __restrict__ Ua, const double* __restrict__ sig_b,
                                                      const c128* __restrict__ Ub, const double* __restrict__ thr,
                                                      double* __restrict__ partial) {
    __shared__ c128 ta[DT][DT + 1], tb[DT][DT + 1];
    __shared__ double sh[32];
    const long long i0 = (long long)blockIdx.y * DT, j0 = (long long)blockIdx.x * DT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 32
    c128 acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = mk<double>(0.0, 0.0);
    for (long long r0 = 0; r0 < n; r0 += DT) {
        for (int q = ty; q < DT; q += 8) {
            const long long i = i0 + q, j = j0 + q, r = r0 + tx;
            ta[q][tx] = (i < n && r < n) ? Ua[i * n + r] : mk<double>(0.0, 0.0);
            tb[q][tx] = (j < n && r < n) ? Ub[j * n + r] : mk<double>(0.0, 0.0);
        }
        __syncthreads();
        // thread (ty, tx): rows i = ty + 8q of the tile, column j = tx
#pragma unroll
        for (int q = 0; q < 4; ++q)
            for (int k = 0; k < DT; ++k) cmacc(acc[q], ta[ty + 8 * q][k], tb[tx][k]);
        __syncthreads();
    }
    const double ta0 = thr[0], tb0 = thr[1];
    double s = 0.0;
    const long long j = j0 + tx;
    const double bj = j < n ? keep_inv(sig_b[j], tb0) : 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long i = i0 + ty + 8 * q;
        if (i < n) s += keep_inv(sig_a[i], ta0) * bj * cabs2(acc[q]);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partial[(long long)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// out = {F, eps_F, kappa(A), kappa(B), r_lambda} from the partial sums and the ascending spectra
__global__ void __launch_bounds__(256) diag_final_kernel(long long n, const double* __restrict__ ev_a,
                                                         const double* __restrict__ ev_b,
                                                         const double* __restrict__ thr,
                                                         const double* __restrict__ partial, long long npart,
                                                         double* __restrict__ out) {
    __shared__ double sh[32];
    double tr = 0.0;
    for (long long k = threadIdx.x; k < npart; k += blockDim.x) tr += partial[k];
    tr = block_sum(tr, sh);
    // spectra of A and B in descending order: a_desc[k] = keep/s_a,asc[k'] over the kept
    // eigenvalues in ascending order of s, then zeros for the cut ones
    const double ta = thr[0], tb = thr[1];
    long long ca = 0, cb = 0;  // number cut
    for (long long k = threadIdx.x; k < n; k += blockDim.x) {
        ca += ev_a[k] > ta ? 0 : 1;
        cb += ev_b[k] > tb ? 0 : 1;
    }
    ca = (long long)block_sum((double)ca, sh);
    cb = (long long)block_sum((double)cb, sh);
    auto a_desc = [&](long long k) { return k < n - ca ? 1.0 / ev_a[ca + k] : 0.0; };
    auto b_desc = [&](long long k) { return k < n - cb ? 1.0 / ev_b[cb + k] : 0.0; };
    double sa = 0.0, sb = 0.0, saa = 0.0, sbb = 0.0, sab = 0.0;
    for (long long k = threadIdx.x; k < n; k += blockDim.x) {
        const double x = a_desc(k), y = b_desc(k);
        sa += x;
        sb += y;
        saa += x * x;
        sbb += y * y;
        sab += x * y;
    }
    sa = block_sum(sa, sh);
    sb = block_sum(sb, sh);
    saa = block_sum(saa, sh);
    sbb = block_sum(sbb, sh);
    sab = block_sum(sab, sh);
    if (threadIdx.x != 0) return;
    const double nn = (double)n;
    const double cov = sab - sa * sb / nn, va = saa - sa * sa / nn, vb = sbb - sb * sb / nn;
    out[0] = tr / sqrt(saa * sbb);
    out[1] = sqrt(fmax(saa + sbb - 2.0 * tr, 0.0)) / sqrt(sbb);
    out[2] = (n - ca > 0) ? (1.0 / ev_a[ca]) / (1.0 / ev_a[n - 1]) : 0.0;
    out[3] = (n - cb > 0) ? (1.0 / ev_b[cb]) / (1.0 / ev_b[n - 1]) : 0.0;
    out[4] = cov / sqrt(va * vb);
}

}  // namespace

cudaError_t launch_born_weights(const c128* logpsi, long long n, double* w, cudaStream_t st) {
    count_launch();
    born_weights_kernel<<<1, 1024, 0, st>>>(logpsi, n, w);
    return cudaGetLastError();
}

cudaError_t launch_block_restrict(const c128* S, long long n, const int64_t* block_off, int nb, c128* out,
                                  long long* blk_of, cudaStream_t st) {
    if (nb < 1 || nb > MAXB) return cudaErrorInvalidValue;
    OffTab off;
    for (int b = 0; b <= nb; ++b) off.v[b] = block_off[b];
    count_launch();
    block_index_kernel<<<nb, 256, 0, st>>>(off, nb, blk_of);
    count_launch();
    block_restrict_kernel<<<1024, 256, 0, st>>>(S, n, blk_of, out);
    return cudaGetLastError();
}

cudaError_t launch_inverse_diagnostics(long long n, const double* sig_a, const double* ev_a, const c128* Ua,
                                       const double* sig_b, const double* ev_b, const c128* Ub, double cutoff,
                                       int mode, double* partial, double* out, cudaStream_t st) {
    double* thr = partial;  // two words, then the tile partials
    count_launch();
    thresholds_kernel<<<1, 32, 0, st>>>(ev_a, ev_b, n, cutoff, mode, thr);
    const unsigned T = (unsigned)((n + DT - 1) / DT);
    count_launch();
    overlap_kernel<<<dim3(T, T), 256, 0, st>>>(n, sig_a, Ua, sig_b, Ub, thr, partial + 2);
    count_launch();
    diag_final_kernel<<<1, 256, 0, st>>>(n, ev_a, ev_b, thr, partial + 2, (long long)T * T, out);
    return cudaGetLastError();
}

}  // namespace nqs
