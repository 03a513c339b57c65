// Block-layer QGT on CUDA cores (FP64 and FP32 paths), Eq. 3:
//   S_b[k][l] = sum_s w_s conj(dO_k(s)) dO_l(s),   k, l in block b, k >= l.
// Operands are the parameter-major centred rows (contiguous samples), so a
// 64 x 64 complex output tile streams two 64-row panels along the sample axis
// through shared memory; each thread owns a 4 x 4 register tile. Only
// lower-triangle tiles are launched (the QGT is Hermitian). In FP32 the partial
// sums of each 16-sample stage are folded into FP64 accumulators, so the
// accumulation error does not grow with the number of samples.
#include "internal.cuh"

namespace nqs {

constexpr int GT = 64;   // complex output tile
constexpr int GK = 16;   // samples per shared-memory stage

void gram_table(const int64_t* block_off, int nb, int tile_rows, GramTable* tab) {
    tab->nb = nb;
    tab->group = 1;
    long long tiles = 0, soff = 0;
    for (int b = 0; b < nb; ++b) {
        const long long n = block_off[b + 1] - block_off[b];
        const long long T = (n + tile_rows - 1) / tile_rows;
        tab->b[b].row0 = block_off[b];
        tab->b[b].s_off = soff;
        tab->b[b].n = (int)n;
        tab->b[b].tiles = (int)(T * (T + 1) / 2);
        tab->b[b].tile0 = tiles;
        tab->b[b].scale = 0.0;
        tiles += T * (T + 1) / 2;
        soff += n * n;
    }
    tab->total_tiles = tiles;
}

__device__ __forceinline__ void tile_coords(const GramTable& tab, long long t, int* b, int* I, int* J) {
    int lo = 0, hi = tab.nb - 1;
    while (lo < hi) {  // last block with tile0 <= t
        const int mid = (lo + hi + 1) >> 1;
        if (tab.b[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    *b = lo;
    const long long r = t - tab.b[lo].tile0;
    long long i = (long long)((sqrt(8.0 * (double)r + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) / 2 <= r) ++i;
    while (i * (i + 1) / 2 > r) --i;
    *I = (int)i;
    *J = (int)(r - i * (i + 1) / 2);
}

template <typename R>
__global__ void __launch_bounds__(256) gram_simt_kernel(const cx<R>* __restrict__ dO, long long ldo, long long ns,
                                                         const double* __restrict__ w, double scale,
                                                         const __grid_constant__ GramTable tab,
                                                         c128* __restrict__ S) {
    __shared__ cx<R> As[GK][GT + 1];
    __shared__ cx<R> Bs[GK][GT + 1];
    int b, I, J;
    tile_coords(tab, blockIdx.x, &b, &I, &J);
    const GBlk blk = tab.b[b];
    const int n = blk.n;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    c128 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = mk<double>(0.0, 0.0);
    const long long rowA = blk.row0 + (long long)I * GT;
    const long long rowB = blk.row0 + (long long)J * GT;
    for (long long s0 = 0; s0 < ns; s0 += GK) {
        for (int idx = threadIdx.x; idx < GT * GK; idx += blockDim.x) {
            const int r = idx / GK, k = idx % GK;
            const long long s = s0 + k;
            cx<R> va = mk<R>(R(0), R(0)), vb = mk<R>(R(0), R(0));
            if (s < ns) {
                if (I * GT + r < n) va = dO[(rowA + r) * ldo + s];
                if (J * GT + r < n) vb = dO[(rowB + r) * ldo + s];
                if (w) {
                    const R ws = (R)w[s];
                    va = ws * va;
                }
            }
            As[k][r] = va;
            Bs[k][r] = vb;
        }
        __syncthreads();
        cx<R> part[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) part[a][c] = mk<R>(R(0), R(0));
#pragma unroll
        for (int k = 0; k < GK; ++k) {
            cx<R> av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[k][ty + 16 * a];
#pragma unroll
            for (int c = 0; c < 4; ++c) bv[c] = Bs[k][tx + 16 * c];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) cmacc(part[a][c], av[a], bv[c]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] = acc[a][c] + ccast<double>(part[a][c]);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int k = I * GT + ty + 16 * a;
        if (k >= n) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int l = J * GT + tx + 16 * c;
            if (l >= n) continue;
            const double sc = blk.scale > 0.0 ? blk.scale : scale;
            S[blk.s_off + (long long)k * n + l] = mk<double>(sc * acc[a][c].re, sc * acc[a][c].im);
        }
    }
}

cudaError_t launch_gram_simt(int prec, const void* dO, long long ldo, long long ns, const double* w,
                             double scale, const GramTable& tab, c128* S, cudaStream_t st) {
    if (tab.total_tiles <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)tab.total_tiles;
    if (prec == NQS_FP64) {
        count_launch();
        gram_simt_kernel<double><<<grid, 256, 0, st>>>((const c128*)dO, ldo, ns, w, scale, tab, S);
    } else {
        count_launch();
        gram_simt_kernel<float><<<grid, 256, 0, st>>>((const c64*)dO, ldo, ns, w, scale, tab, S);
    }
    return cudaGetLastError();
}

}  // namespace nqs
