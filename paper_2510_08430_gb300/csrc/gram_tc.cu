// Block-layer QGT on the 5th-generation tensor cores (tcgen05), split BF16 (Eq. 3):
//   S_b = sum_s w_s dO_b(s)^H dO_b(s)
// computed as the real Gram G = X X^T of the interleaved real rows X[2k] = Re dO_k,
// X[2k+1] = Im dO_k (samples contiguous, i.e. K-major operands), so that
//   Re S[k][l] = G[2k][2l] + G[2k+1][2l+1],   Im S[k][l] = G[2k][2l+1] - G[2k+1][2l].
// Every entry is split into BF16 terms x = x1 + x2 (+ x3 (+ x4)) and G is accumulated
// from the leading products x1 y1 (accumulator A0) and the correction products
// (accumulator A1). Two splits: element-wise (each term the BF16 rounding of the
// remainder, 2 or 3 terms), and grouped error-free (per parameter and 32-sample group
// a common power of two, five slices of at most 8-bit integers; Ozaki, Ogita, Oishi
// and Rump 2012), in which the A0 sums and the order-1 sums are exact. FP32 accumulation in tensor memory
// spans at most one K block; the epilogue folds every work item into double-float
// (FP32 hi + lo, TwoSum) running sums of A0 and FP32 sums of A1 held in registers,
// so the accumulation error does not grow with the number of samples. S is written
// in FP64 once per tile.
//
// Persistent kernel, one CTA per SM, static round-robin over the lower-triangle
// 128 x 128 tiles of every block. Warp roles: warp 0 issues TMA loads (128B
// swizzle) into a STAGES-deep ring, warp 1 allocates tensor memory and issues
// tcgen05.mma, warps 2-9 (two per tensor-memory lane quarter, one per 64-column
// half of the tile) drain the double-buffered accumulator pairs
// (tcgen05.ld), combine the 2 x 2 real blocks into complex entries and fold
// them. Every mbarrier wait is bounded; on expiry the kernel records
// NQS_ERR_TIMEOUT, drains its own copies and MMAs, frees tensor memory and
// returns.
#include <cstdlib>
#include <new>
#include <cuda.h>
#include <cuda_bf16.h>
#include "internal.cuh"

namespace nqs {

namespace tc {

constexpr int BM = 128;          // real rows per tile (64 complex)
constexpr int BK = 64;           // samples of one K block (128-byte swizzle rows)
constexpr int NTHREADS = 320;                    // TMA warp, MMA warp, 8 epilogue warps
constexpr int NEPI = 256;                        // epilogue threads
constexpr uint32_t TMEM_COLS = 512;              // 2 buffers x up to 2 accumulators x 128 columns
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s budget per wait

// NPL planes per operand; NPROD products (plane of A, plane of B); product 0
// (x1 y1) goes to accumulator A0, all others to A1.
template <int NS> struct Split;
template <> struct Split<2> {   // x1 y1 | x1 y2 + x2 y1
    static constexpr int NPL = 2, NPROD = 3, STAGES = 3;
    __device__ static constexpr int pa(int i) { return i == 2 ? 1 : 0; }
    __device__ static constexpr int pb(int i) { return i == 1 ? 1 : 0; }
};
template <> struct Split<3> {   // x1 y1 | x1 y2 + x2 y1 + x1 y3 + x3 y1 + x2 y2
    static constexpr int NPL = 3, NPROD = 6, STAGES = 2;
    __device__ static constexpr int pa(int i) { return i == 2 ? 1 : (i == 4 ? 2 : (i == 5 ? 1 : 0)); }
    __device__ static constexpr int pb(int i) { return i == 1 ? 1 : (i == 3 ? 2 : (i == 5 ? 1 : 0)); }
};

// Grouped error-free slices, five per value: s1 s1 -> A0; into A1 first every product of
// order 2..4 (issued while A1 is small), then the order-1 products s1 s2 + s2 s1 (exact).
template <> struct Split<5> {
    static constexpr int NPL = 5, NPROD = 15, STAGES = 2;
    // 0:(0,0) | 1:(0,2) 2:(2,0) 3:(1,1) 4:(0,3) 5:(3,0) 6:(1,2) 7:(2,1) 8:(0,4) 9:(4,0) 10:(1,3)
    //          11:(3,1) 12:(2,2) 13:(0,1) 14:(1,0)
    __device__ static constexpr int pa(int i) {
        return i == 2 ? 2 : i == 3 ? 1 : i == 5 ? 3 : i == 6 ? 1 : i == 7 ? 2 : i == 9 ? 4 : i == 10 ? 1
             : i == 11 ? 3 : i == 12 ? 2 : i == 14 ? 1 : 0;
    }
    __device__ static constexpr int pb(int i) {
        return i == 1 ? 2 : i == 3 ? 1 : i == 4 ? 3 : i == 6 ? 2 : i == 7 ? 1 : i == 8 ? 4 : i == 10 ? 3
             : i == 11 ? 1 : i == 12 ? 2 : i == 13 ? 1 : 0;
    }
};

// Packed pairs of FP32 numbers (here: the real and imaginary part of one output), operated on
// by the two-lane FP32 instructions of sm_100-class GPUs with round-to-nearest in each lane.
__device__ __forceinline__ uint64_t pk2(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(uint64_t r, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// (s, e) with s + e = a + b exactly, lane by lane (TwoSum, Knuth)
__device__ __forceinline__ void two_sum2(uint64_t a, uint64_t b, uint64_t& s, uint64_t& e) {
    s = add2(a, b);
    const uint64_t bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}


__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// try_wait that may suspend the thread in hardware for up to `ns` nanoseconds while the
// phase is incomplete (a waiting warp then takes no issue slots from the working ones)
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
// Bounded wait: false on timeout or (if abort_flag is not NULL) when another
// role has aborted. Each try suspends for at most 20 us; the iteration cap backs up the
// time budget.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
        if (abort_flag && *abort_flag) return false;
        if (gtimer() - t0 > WAIT_NS) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

// Shared-memory matrix descriptor: K-major, rows of KB BF16 (128-byte swizzle for
// KB = 64, 64-byte swizzle for KB = 32), 8-row core groups 8 * 2 KB bytes apart
// (SBO), descriptor version 1, leading offset unused (1).
template <int KB>
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    static_assert(KB == 64 || KB == 32, "K block of 32 or 64 BF16");
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;                          // LBO (ignored for swizzled K-major)
    d |= (uint64_t)((8u * 2u * KB) >> 4) << 32;       // SBO
    d |= (uint64_t)1u << 46;                          // version
    d |= (uint64_t)(KB == 64 ? 2u : 4u) << 61;        // SWIZZLE_128B / SWIZZLE_64B
    return d;
}

// Shared-memory descriptor of slice `pl` at MMA K-step kk within one operand's part of a stage.
// Element-wise splits (PAIRED false): pl-th tile of 128 rows x KB BF16. Grouped split (PAIRED):
// a 16 KB tile of 128-byte rows holding slices 1-2 (32 samples each, 128-byte swizzle), one
// holding slices 3-4, and an 8 KB tile of slice 5 (64-byte rows, 64-byte swizzle); a slice's
// K-steps start 32 bytes apart inside its half of the row.
template <bool PAIRED, int KB>
__device__ __forceinline__ uint64_t plane_desc(uint32_t side, int pl, int kk) {
    if (PAIRED) {
        if (pl < 4) return sdesc<64>(side + (uint32_t)((pl >> 1) * (BM * 128) + (pl & 1) * 64 + kk * 32));
        return sdesc<32>(side + (uint32_t)(2 * BM * 128 + kk * 32));
    }
    return sdesc<KB>(side + (uint32_t)(pl * (BM * KB * 2) + kk * 32));
}

// Instruction descriptor, kind::f16: D FP32, A/B BF16, both K-major, M = 128, N = 128.
__host__ __device__ constexpr uint32_t idesc_bf16_128x128() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TileInfo {
    int b, I, J;
};

__device__ __forceinline__ void tri_decode(long long r, long long* I, long long* J) {
    long long i = (long long)((sqrt(8.0 * (double)r + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) / 2 <= r) ++i;
    while (i * (i + 1) / 2 > r) --i;
    *I = i;
    *J = r - i * (i + 1) / 2;
}

// Tile t of the launch -> (block, I, J), J <= I. Within a block the lower-triangle tiles are
// taken in square groups of G x G (G = tab.group): super-rows of G tile rows in turn; in each,
// the off-diagonal G x G groups left to right (row-major inside), then the diagonal group's
// lower triangle. Consecutive tiles (the CTAs running at the same time) then share G row panels
// and G column panels, which stay in L2 while they stream the samples. G = 1 is row by row.
__device__ __forceinline__ TileInfo decode(const GramTable& tab, long long t) {
    int lo = 0, hi = tab.nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab.b[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    const long long r = t - tab.b[lo].tile0;
    const long long G = tab.group > 0 ? tab.group : 1;
    const long long T = (tab.b[lo].n + BM / 2 - 1) / (BM / 2);  // tile rows of the block
    // super-row S (rows S G .. S G + h - 1, h = min(G, T - S G)) holds h S G + h (h + 1) / 2 tiles;
    // every super-row before the last has h = G
    long long Sr = 0, base = 0;
    for (;;) {
        const long long h = (T - Sr * G) < G ? (T - Sr * G) : G;
        const long long cnt = h * Sr * G + h * (h + 1) / 2;
        if (r < base + cnt || h < G) break;  // the last super-row has h <= G
        base += cnt;
        ++Sr;
    }
    const long long h = (T - Sr * G) < G ? (T - Sr * G) : G;
    const long long u = r - base;
    TileInfo ti;
    ti.b = lo;
    if (u < h * Sr * G) {       // off-diagonal group J' = u / (h G), row-major inside
        const long long Jg = u / (h * G), loc = u % (h * G);
        ti.I = (int)(Sr * G + loc / G);
        ti.J = (int)(Jg * G + loc % G);
    } else {                    // diagonal group: lower triangle of h x h
        long long i, j;
        tri_decode(u - h * Sr * G, &i, &j);
        ti.I = (int)(Sr * G + i);
        ti.J = (int)(Sr * G + j);
    }
    return ti;
}

struct Maps {
    CUtensorMap m[5];
};

// Work item = (tile, kpi MMA K-steps of 16 samples; kpi divides KB / 16). Each work item
// owns one of two accumulator pairs (A0, A1) in tensor memory; smem stages hold
// one 64-sample K block each.
// KB: samples per K block (64 or 32). GROUPED: every group of GRAM_GROUP = KB samples carries
// its own per-parameter exponents gexp[group][param]; the epilogue scales each group by
// 2^(E_k + E_l) (one work item per group and smem stage, kpi = KB / 16 MMA K-steps).
template <int NSPLIT, bool GROUPED, int KB>
__global__ void __launch_bounds__(NTHREADS, 1)
    gram_tc_kernel(const __grid_constant__ Maps maps, const __grid_constant__ GramTable tab, int nkb, int kpi,
                   double scale, const int8_t* __restrict__ gexp, long long np, c128* __restrict__ S,
                   DevStatus* status) {
    using SP = Split<NSPLIT>;
    constexpr int NS = SP::NPL;
    constexpr int STAGES = SP::STAGES;
    constexpr int KTILE_BYTES = BM * KB * 2;
    constexpr int STAGE_BYTES = 2 * NS * KTILE_BYTES;
    constexpr int KSTEPS = KB / 16;
    constexpr uint32_t BUF_COLS = 256u;  // A0 and A1, 128 columns each
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* ring = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], tfull_bar[2], tempty_bar[2], done_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull_bar[a], 1);
            mbar_init(&tempty_bar[a], NEPI);
        }
        mbar_init(&done_bar, 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem_base = tmem_base_sh;
    volatile int* abort_flag = &abort_sh;
    const long long total = tab.total_tiles;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            for (int p = 0; p < (GROUPED ? 3 : NS); ++p)
                asm volatile("prefetch.tensormap [%0];" ::"l"(&maps.m[p]) : "memory");
            uint32_t q = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
                const TileInfo ti = decode(tab, t);
                const GBlk blk = tab.b[ti.b];
                const int rowA = (int)(2 * blk.row0 + (long long)ti.I * BM);
                const int rowB = (int)(2 * blk.row0 + (long long)ti.J * BM);
                const bool diag = ti.I == ti.J;
                for (int kb = 0; kb < nkb; ++kb, ++q) {
                    const int s = q % STAGES;
                    const uint32_t ph = (q / STAGES) & 1u;
                    if (!mbar_wait(&empty_bar[s], ph ^ 1u, abort_flag)) { ok = false; break; }
                    unsigned char* st = ring + (size_t)s * STAGE_BYTES;
                    mbar_expect_tx(&full_bar[s], (diag ? NS : 2 * NS) * KTILE_BYTES);
                    if (GROUPED) {  // three boxes per operand: slices 1-2, 3-4 (128-byte rows), 5
                        for (int o = 0; o < (diag ? 1 : 2); ++o) {
                            unsigned char* side = st + o * NS * KTILE_BYTES;
                            const int row = o ? rowB : rowA;
                            tma_load_2d(side, &maps.m[0], &full_bar[s], kb * 2 * KB, row);
                            tma_load_2d(side + BM * 128, &maps.m[1], &full_bar[s], kb * 2 * KB, row);
                            tma_load_2d(side + 2 * BM * 128, &maps.m[2], &full_bar[s], kb * KB, row);
                        }
                    } else {
                        for (int p = 0; p < NS; ++p)
                            tma_load_2d(st + p * KTILE_BYTES, &maps.m[p], &full_bar[s], kb * KB, rowA);
                        if (!diag)
                            for (int p = 0; p < NS; ++p)
                                tma_load_2d(st + (NS + p) * KTILE_BYTES, &maps.m[p], &full_bar[s], kb * KB, rowB);
                    }
                }
            }
            if (!ok) {
                *abort_flag = 1;
                set_status(status, NQS_ERR_TIMEOUT, W_GRAM_TC, 0);
            }
            // drain: the last issued phase of every stage must have landed before exit
            for (uint32_t st = 0; st < (uint32_t)STAGES; ++st) {
                if (q > st) {
                    const uint32_t last = st + (uint32_t)STAGES * ((q - 1u - st) / (uint32_t)STAGES);
                    mbar_wait(&full_bar[st], (last / STAGES) & 1u, nullptr);
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_128x128();
            const int nsub = KSTEPS / kpi;
            uint32_t q = 0, w = 0;  // smem stage counter, accumulator work-item counter
            bool ok = true;
            for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
                const TileInfo ti = decode(tab, t);
                const bool diag = ti.I == ti.J;
                for (int kb = 0; kb < nkb && ok; ++kb, ++q) {
                    const int s = q % STAGES;
                    const uint32_t ph = (q / STAGES) & 1u;
                    if (!mbar_wait(&full_bar[s], ph, abort_flag)) { ok = false; break; }
                    fence_after();
                    const uint32_t base = smem_u32(ring + (size_t)s * STAGE_BYTES);
                    const uint32_t boff = diag ? 0u : (uint32_t)(NS * KTILE_BYTES);
                    for (int sub = 0; sub < nsub; ++sub, ++w) {
                        const uint32_t acc = w & 1u;
                        const uint32_t tmem_d = tmem_base + acc * BUF_COLS;
                        if (!mbar_wait(&tempty_bar[acc], ((w >> 1) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
                        fence_after();
                        // product-major over the item's K-steps: every small product enters A1
                        // before the large order-1 ones (Split<5> lists them last)
#pragma unroll
                        for (int pr = 0; pr < SP::NPROD; ++pr) {
                            for (int kk = sub * kpi; kk < (sub + 1) * kpi; ++kk) {
                                // 16 BF16 = 32 bytes per K-step inside the swizzle row
                                const uint64_t ad = plane_desc<GROUPED, KB>(base, SP::pa(pr), kk);
                                const uint64_t bd = plane_desc<GROUPED, KB>(base + boff, SP::pb(pr), kk);
                                // product 0 -> A0; products 1.. -> A1; the first write of each resets it
                                const uint32_t first = (kk == sub * kpi && pr <= 1) ? 0u : 1u;
                                umma(tmem_d + (pr == 0 ? 0u : 128u), ad, bd, idesc, first);
                            }
                        }
                        umma_commit(&tfull_bar[acc]);   // hands the accumulator pair to the epilogue
                    }
                    if (!ok) break;
                    umma_commit(&empty_bar[s]);     // frees the smem stage when these MMAs complete
                }
            }
            if (!ok) {
                *abort_flag = 1;
                set_status(status, NQS_ERR_TIMEOUT, W_GRAM_TC, 1);
            }
            // wait for every MMA issued by this thread before tensor memory is freed
            umma_commit(&done_bar);
            mbar_wait(&done_bar, 0u, nullptr);
        }
    } else {
        // ---------------- epilogue: warp w owns TMEM lane quarter w % 4 and column half (w - 2) / 4
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;   // 64 real columns = 32 complex columns each
        const int r = quarter * 32 + lane;  // accumulator row (real row within the tile)
        const int cpar = r & 1;             // 0: Re row, 1: Im row of complex row r/2
        uint32_t q = 0;
        bool ok = true;
        const int nitems = nkb * (KSTEPS / kpi);
        for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
            const TileInfo ti = decode(tab, t);
            const GBlk blk = tab.b[ti.b];
            const int n = blk.n;
            const long long k = (long long)ti.I * (BM / 2) + (r >> 1);
            // double-float running sums of the 16 complex outputs this lane owns, renormalised
            // after every work item
            // (Re, Im) packed: high words hw[j], low words lw[j]
            uint64_t hw[16], lw[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) hw[j] = lw[j] = 0ull;
            for (int item = 0; item < nitems; ++item, ++q) {
                const uint32_t acc = q & 1u;
                if (!mbar_wait(&tfull_bar[acc], (q >> 1) & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                fence_after();
                // grouped mode: exponents of this group of kpi * 16 samples (row k, this lane's columns)
                int ekg = 0;
                const int8_t* gcol = nullptr;
                if (GROUPED) {
                    const int8_t* ge = gexp + (long long)item * np + blk.row0;
                    ekg = (k < n) ? (int)ge[k] : 0;
                    gcol = ge + (long long)ti.J * (BM / 2) + 32 * half;
                }
#pragma unroll
                for (int chunk = 0; chunk < 8; ++chunk) {
                    uint32_t v0[8], v1[8];
                    const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + acc * BUF_COLS +
                                           (uint32_t)(64 * half + 8 * chunk);
                    tmem_ld8(taddr, v0);
                    tmem_ld8(taddr + 128u, v1);
                    // 8 real columns = 2 pairs of complex columns (l0 = 2m, l1 = 2m + 1)
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        float re0, im0, re1, im1;
                        {
                            // A0: in grouped mode these are exact sums on a common grid, so the
                            // 2 x 2 combination below is exact in FP32
                            const float g0 = __uint_as_float(v0[4 * m + 0]);  // col (l0, re)
                            const float g1 = __uint_as_float(v0[4 * m + 1]);  // col (l0, im)
                            const float g2 = __uint_as_float(v0[4 * m + 2]);  // col (l1, re)
                            const float g3 = __uint_as_float(v0[4 * m + 3]);  // col (l1, im)
                            // even lane (Re row) sends its l1 pair, odd lane (Im row) its l0 pair
                            const float y0 = __shfl_xor_sync(0xffffffffu, cpar ? g0 : g2, 1);
                            const float y1 = __shfl_xor_sync(0xffffffffu, cpar ? g1 : g3, 1);
                            if (cpar == 0) {   // S[k][l0]: g00 = g0, g01 = g1, g10 = y0, g11 = y1
                                re0 = g0 + y1;
                                im0 = g1 - y0;
                            } else {           // S[k][l1]: g00 = y0, g01 = y1, g10 = g2, g11 = g3
                                re0 = y0 + g3;
                                im0 = y1 - g2;
                            }
                        }
                        {
                            const float g0 = __uint_as_float(v1[4 * m + 0]);
                            const float g1 = __uint_as_float(v1[4 * m + 1]);
                            const float g2 = __uint_as_float(v1[4 * m + 2]);
                            const float g3 = __uint_as_float(v1[4 * m + 3]);
                            const float y0 = __shfl_xor_sync(0xffffffffu, cpar ? g0 : g2, 1);
                            const float y1 = __shfl_xor_sync(0xffffffffu, cpar ? g1 : g3, 1);
                            if (cpar == 0) {
                                re1 = g0 + y1;
                                im1 = g1 - y0;
                            } else {
                                re1 = y0 + g3;
                                im1 = y1 - g2;
                            }
                        }
                        const int j = 2 * chunk + m;
                        uint64_t v0 = pk2(re0, im0), v1 = pk2(re1, im1);
                        if (GROUPED) {
                            const long long lcol = (long long)ti.J * (BM / 2) + 32 * half + 2 * j + cpar;
                            const int el = (lcol < n) ? (int)gcol[2 * j + cpar] : 0;
                            const int es = ekg + el;  // 2^(E_k + E_l), exact
                            const float f = (es >= -126 && es <= 127) ? __int_as_float((es + 127) << 23)
                                                                      : ldexpf(1.f, es);
                            const uint64_t ff = pk2(f, f);
                            v0 = mul2(v0, ff);
                            v1 = mul2(v1, ff);
                        }
                        // (h, l) += v0 (exact) + v1: TwoSum of the high word with the exact
                        // leading part, then renormalise with the small terms so that the low
                        // word never accumulates across groups (Re and Im in one packed pair)
                        uint64_t sh, se;
                        two_sum2(hw[j], v0, sh, se);
                        two_sum2(sh, add2(add2(se, v1), lw[j]), hw[j], lw[j]);
                    }
                }
                fence_before();
                mbar_arrive(&tempty_bar[acc]);
            }
            if (!ok) break;
            if (k < n) {
                c128* Srow = S + blk.s_off + k * n;
                const double sc = blk.scale > 0.0 ? blk.scale : scale;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const long long l = (long long)ti.J * (BM / 2) + 32 * half + 2 * j + cpar;
                    float hre, him, lre, lim;
                    upk2(hw[j], hre, him);
                    upk2(lw[j], lre, lim);
                    if (l < n)
                        Srow[l] = mk<double>(sc * ((double)hre + (double)lre), sc * ((double)him + (double)lim));
                }
            }
        }
        if (!ok) {
            *abort_flag = 1;
            set_status(status, NQS_ERR_TIMEOUT, W_GRAM_TC, 2);
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
    }
}

}  // namespace tc

cudaError_t launch_gram_tc_tab(int nsplit, const void* const* planes, const int8_t* gexp, long long np,
                               long long rows, long long ldk, long long kpad, double scale, const GramTable& tab,
                               c128* S, DevStatus* status, cudaStream_t st);

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

static bool make_map(CUtensorMap* m, const void* base, long long rows, long long ldk, int kb) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ldk * 2};
    cuuint32_t box[2] = {(cuuint32_t)kb, (cuuint32_t)tc::BM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, kb == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int NSPLIT, bool GROUPED, int KB>
static cudaError_t launch_tc(const tc::Maps& maps, const GramTable& tab, long long kpad, int kpi, double scale,
                            const int8_t* gexp, long long np, c128* S, DevStatus* status, int sms, cudaStream_t st) {
    const size_t smem = (size_t)tc::Split<NSPLIT>::STAGES * 2 * tc::Split<NSPLIT>::NPL * (tc::BM * KB * 2) + 1024;
    cudaError_t e = cudaFuncSetAttribute(tc::gram_tc_kernel<NSPLIT, GROUPED, KB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long grid = tab.total_tiles < sms ? tab.total_tiles : sms;
    count_launch();
    tc::gram_tc_kernel<NSPLIT, GROUPED, KB><<<(unsigned)grid, tc::NTHREADS, smem, st>>>(
        maps, tab, (int)(kpad / KB), kpi, scale, gexp, np, S, status);
    return cudaGetLastError();
}

cudaError_t launch_gram_tc(int nsplit, const void* const* planes, const int8_t* gexp, long long np, long long rows,
                           long long ldk, long long kpad, double scale, const GramTable& tab_in, c128* S,
                           DevStatus* status, cudaStream_t st) {
    // the tile-group edge of this call from the tuning table (largest block, samples summed)
    GramTable* tabp = new (std::nothrow) GramTable(tab_in);
    if (!tabp) return cudaErrorMemoryAllocation;
    long long max_nb = 0;
    for (int b = 0; b < tabp->nb; ++b) max_nb = tabp->b[b].n > max_nb ? tabp->b[b].n : max_nb;
    tabp->group = gram_group_edge(max_nb, kpad);
    const cudaError_t e = launch_gram_tc_tab(nsplit, planes, gexp, np, rows, ldk, kpad, scale, *tabp, S, status, st);
    delete tabp;
    return e;
}

cudaError_t launch_gram_tc_tab(int nsplit, const void* const* planes, const int8_t* gexp, long long np,
                               long long rows, long long ldk, long long kpad, double scale, const GramTable& tab,
                               c128* S, DevStatus* status, cudaStream_t st) {
    static int kpi = -1;  // MMA K-steps per accumulator flush (1, 2 or 4); NQS_GRAM_KPI overrides
    if (kpi < 0) {
        const char* env = getenv("NQS_GRAM_KPI");
        const int v = env ? atoi(env) : GRAM_KPI_DEFAULT;
        kpi = (v == 1 || v == 2 || v == 4) ? v : GRAM_KPI_DEFAULT;
    }
    if (tab.total_tiles <= 0) return cudaSuccess;
    if (nsplit != 2 && nsplit != 3 && nsplit != 5) return cudaErrorInvalidValue;
    int dev = 0;
    cudaGetDevice(&dev);
    int major = 0, minor = 0, sms = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (major != 10 || minor != 3) return cudaErrorNotSupported;
    if (ldk % tc::BK != 0 || kpad % tc::BK != 0 || kpad > ldk) return cudaErrorInvalidValue;
    const int kb = nsplit == 5 ? 32 : 64;
    tc::Maps maps;
    for (int p = 0; p < plane_units(nsplit); ++p) {
        if (reinterpret_cast<uintptr_t>(planes[p]) & 15) return cudaErrorInvalidValue;
        // grouped split: units of slices 1-2 and 3-4 have rows of 2 ldk read in 64-element
        // (128-byte) boxes; slice 5 rows of ldk in 32-element boxes
        const long long len = plane_row_len(nsplit, p, ldk);
        const int box = (nsplit == 5 && p < 2) ? 64 : kb;
        if (!make_map(&maps.m[p], planes[p], rows, len, box)) return cudaErrorInvalidValue;
    }
    if (nsplit == 2) return launch_tc<2, false, 64>(maps, tab, kpad, kpi, scale, nullptr, np, S, status, sms, st);
    if (nsplit == 3) return launch_tc<3, false, 64>(maps, tab, kpad, kpi, scale, nullptr, np, S, status, sms, st);
    // one work item per exponent group = one 32-sample K block (two MMA K-steps)
    static_assert(GRAM_GROUP == 32, "an exponent group is one smem stage of the grouped kernel");
    return launch_tc<5, true, 32>(maps, tab, kpad, GRAM_GROUP / 16, scale, gexp, np, S, status, sms, st);
}

}  // namespace nqs
