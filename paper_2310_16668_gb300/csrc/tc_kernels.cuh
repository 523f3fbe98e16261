// Tensor-core translations for many right-hand sides (FP32_TC precision).
//
// For a work item of up to 128 target rows (rows of one box, or several small
// leaves packed together) the translations are
// U[128 x 32] += G[128 x K] Q[K x 32] over the K source entries of the box's
// tasks, G_ij = G(x_i, y_j) evaluated on the fly, 32 sources per pipeline
// tile. Before the translations of a 32-column pass, tc_bprep_kernel writes
// every source chunk (32 consecutive entries of one box) as one contiguous
// block: its B operand in the MMA's shared-memory layout (K-major, no
// swizzle, 8 x 16-byte core matrices: 512 bytes between core matrices along
// K, 128 bytes between groups of 8 right-hand sides), split into TF32 hi and
// lo, followed by the chunk's coordinates. The CTA is warp-specialised:
//   * warp 8 (producer; lanes fetch 32 tile descriptors at a time, lane 0
//     issues): for tile t it waits until data stage t % 6 is free, arms that
//     stage's "full" mbarrier with the byte count and issues two bulk copies
//     (cp.async.bulk): the source chunk as the prep kernel laid it out (B hi,
//     B lo, coordinates; 9 KB) and the tile descriptor, running up to six
//     tiles ahead of the compute warps;
//   * warp 9, one thread (MMA issuer): for tile m it waits for "A full" and
//     issues 12 tcgen05.mma (kind::tf32, M = 128, N = 32, K = 8: hi*hi +
//     hi*lo + lo*hi for each of 4 K-steps) and commits them to the stage's
//     "empty" mbarrier;
//   * warps 0-7 (compute, two threads per target row, 16 sources each): wait
//     "full", copy their 16 source coordinates once per target slot their
//     rows fall in (one array per axis, warp-private, so only __syncwarp),
//     evaluate the kernel block two sources per paired FP32 instruction
//     (fadd2 / fmul2 / ffma2), split each value into TF32 hi + lo, add the
//     finished accumulator of tile u - 2 into FP32 registers, write A with
//     tcgen05.st (TMEM lane = row, column = source) and arrive on "A full".
// Six data stages and three A buffers keep the bulk copies (issued up to six
// tiles ahead), the kernel evaluation and the tensor core busy at the same
// time; the two accumulator tiles alternate, so each tensor-memory
// accumulation covers one tile only (32 sources) and every longer sum is an
// FP32 round-to-nearest register sum. The dropped lo*lo term and the
// truncation of the lo parts are below 2^-21 of each product.
//
// Masks: a source that a target row's slot must skip (the regrouped
// subtractions of Algorithm 2) gets G = 0 in that row: in that slot's copy of
// the coordinates it sits at 1e30, where r^2 overflows to +inf and the kernel
// value is exactly 0, so the evaluation itself has no per-source test.
// Each half of the compute warps drains 16 of the 32 accumulator columns.
// Waiting threads sleep in the mbarrier (suspend-time hint) rather than spin,
// and every wait is bounded by wall time (globaltimer, 2 s); on timeout the
// kernel raises the status word, keeps the protocol going without hanging,
// waits (bounded) for its copies and MMAs and always frees its tensor memory.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "host.h"
#include "skel_kernels.cuh"

namespace skel {

constexpr int kTpr = 2;                        // compute threads per target row
constexpr int kTcCompute = 128 * kTpr;         // compute threads
constexpr int kSrcPerThread = 32 / kTpr;       // sources of a tile each compute thread evaluates
constexpr int kTcThreads = kTcCompute + 64;    // + the producer warp and the MMA warp
constexpr int kTcN = 32;                       // right-hand sides per pass (MMA N)
constexpr int kTcGroup = 128;                  // tiles summed in registers before the outer sum
constexpr int kNS = 6;                         // data stages (bulk-copy destinations) by default;
                                               // the autotuner may pick 4 or 8 (same arithmetic)
constexpr int kNA = 3;                         // A-operand buffers in tensor memory
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kColD = 0;                  // accumulators D0 [0,32), D1 [32,64)
constexpr uint32_t kColA = 64;                 // A[b]: hi at 64+64b, lo at 96+64b (b < kNA)
constexpr uint32_t kSleepNs = 20000;           // suspend hint of one wait attempt
constexpr uint64_t kWaitLimitNs = 2000000000ull; // a wait gives up after 2 s (TcArgs::wait_ns)

// one source chunk as the prep kernel lays it out in global memory and one
// bulk copy moves it: B hi, B lo, source coordinates (hi, lo)
constexpr int kChunkFloats = 2 * 1024 + 2 * 128;
struct alignas(128) TcStage {
    float bhi[32 * 32];                        // B operand, TF32 hi (bulk-copied, already converted)
    float blo[32 * 32];                        // B operand, TF32 lo
    float4 xh[32];                             // source coordinates (hi)
    float4 xl[32];                             // lo parts (touching-leaf tiles)
    SrcTile tile;                              // 64 B: the tile's descriptor (its own copy)
};
static_assert(offsetof(TcStage, tile) == kChunkFloats * 4, "chunk blob is contiguous in the stage");
// per compute warp: for each target slot its 32 rows touch, the coordinates
// of its kSrcPerThread sources, one array per axis (x, y, z); a source the
// slot skips sits at kFar
constexpr int kWarpSlotFloats = 3 * kSrcPerThread;
constexpr float kFar = 1e30f;                  // r^2 from here overflows to +inf: 1/r = 0
template <int NS>
struct TcShared {
    TcStage st[NS];
    float wc[kTcCompute / 32][kMaxSlots * kWarpSlotFloats];
    float outer[kTcN / kTpr][kTcCompute];      // per compute thread: the sum of its flushed tile groups
    uint64_t full[NS], afull[NS], empty[NS];   // per data stage
    uint32_t tmem;
    uint32_t slots;
};
constexpr int kTcSmemRequest = 112 * 1024;    // at most two CTAs (2 x 256 TMEM columns) per SM
static_assert(sizeof(TcShared<8>) <= kTcSmemRequest, "shared memory plan");

// Stored-operator mode (symmetric store). The rows of every tensor-core item
// are whole source chunks ("row chunks", at most kMaxRc of them); the values
// a tile (item, source chunk c) needs are, for each row chunk a, the block
// G(a, c) of the kernel between the entries of a and of c. For the real
// kernels G(a, c) = G(c, a)^T and the near-field relation is symmetric, so a
// block is stored once, in one orientation, and read directly by one tile and
// transposed by the other. A stored block with R rows and C columns keeps its
// values column by column with an odd pitch P >= R (value (r, j) at
// off + j P + r), so that 32 consecutive rows read 32 consecutive floats and
// the transposed read (r, j) -> off + r P + j, a stride of P, meets every
// shared-memory bank once. Stored values are unmasked; each reader applies
// its own keep mask.
constexpr int kMaxRc = 12;                     // row chunks per item (<= 8 packed leaves + 128 / 32)
constexpr int kSymFloats = (128 + kMaxRc) * 32;  // a stage's block area: row chunk k at (ro_k + k) * 32

struct BlockRef {                              // 16 bytes: one row chunk of one tile
    int64_t off;                               // first float of the stored block
    uint32_t bytes;                            // bulk-copy size (0: no row of this chunk keeps a source)
    uint16_t pitch;                            // P of the stored block
    uint8_t flags;                             // kRefTransposed, kRefRecord
    uint8_t pad;
};
static_assert(sizeof(BlockRef) == 16, "BlockRef is 16 bytes");
constexpr uint8_t kRefTransposed = 1;          // the block is stored as G(c, a): read it transposed
constexpr uint8_t kRefRecord = 2;              // this tile's fill pass writes the block

struct ItemSym {                               // 40 bytes per tensor-core item
    int64_t ref0;                              // its tiles' BlockRefs: ref0 + t * m + k (t = tile of the item)
    int32_t m;                                 // row chunks
    int16_t ro[kMaxRc + 2];                    // first row of each row chunk; ro[m] = nrows
};
static_assert(sizeof(ItemSym) == 40, "ItemSym layout");

struct TcArgs {
    const TcItem* items;
    const SrcTile* tiles;                      // item i's tiles: [list_lo, list_hi) of this array
    const float4* X;
    const float4* Xlo;
    const float* B;                            // per source chunk (kChunkFloats): B hi, B lo, coordinates
    float* U;                                  // entry rows of nrhs (this item's rows are written here)
    float* A;                                  // stored kernel values, or null
    const int64_t* abase;                      // per-tile store: per item, first float of its tiles
    const uint8_t* qmask;                      // per-tile store: per tile, the quads it keeps
    const BlockRef* refs;                      // symmetric store: per tile and row chunk
    const ItemSym* isym;                       // stored-operator mode: per item
    int nrhs;                                  // right-hand sides (row length of U)
    int r0;                                    // first right-hand side of this pass
    float kappa;                               // Helmholtz wavenumber (complex path)
    int* status;
    uint64_t wait_ns;                          // limit of every bounded wait (kWaitLimitNs)
    int withhold_item;                         // test hook: this item's first tile is copied only
                                               // after its consumers gave up waiting (-1: none)
};

__device__ __forceinline__ uint32_t sm_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

// the same test, letting the hardware suspend the thread (up to the hint)
// while the phase is incomplete instead of spinning on issue slots
__device__ __forceinline__ bool mbar_try_sleep(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(ok) : "r"(bar), "r"(parity), "r"(kSleepNs) : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// bounded wait: gives up after limit_ns of wall time
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_sleep(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// Test hook of the bounded waits (TcArgs::withhold_item): before the first
// tile's copies the producer waits until the compute warps have given up
// waiting for them and arrived on "A full"; then it issues the copies and
// waits until they have landed. Every barrier still completes exactly one
// phase per tile, every copy is waited for, and only that tile's values are
// wrong (the kernel raises the status word).
__device__ __forceinline__ bool withhold_first_tile(uint32_t afull0, uint64_t limit_ns) {
    return mbar_wait(afull0, 0u, limit_ns);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// L2 cache policies for the bulk copies: data read once (stored kernel
// blocks, tile descriptors) is evicted first, so that the source chunks' B
// blocks, which every neighbouring item reads again, stay in L2
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void bulk_g2s_hint(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar,
                                              uint64_t policy) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(bar), "l"(policy) : "memory");
}

// B operand layout (K-major, no swizzle): core matrix = 8 right-hand sides x
// 4 sources (16 bytes per row); the 4 groups of 8 right-hand sides of one
// 4-source slab are contiguous (SBO = 128 B) and slabs follow along K
// (LBO = 512 B): element (n, j) at byte (j/4)*512 + n*16 + (j%4)*4.
constexpr uint32_t kBLbo = 512, kBSbo = 128;

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((kBLbo >> 4) & 0x3FFF) << 16;   // LBO: next core matrix along K
    d |= (uint64_t)((kBSbo >> 4) & 0x3FFF) << 32;   // SBO: next group of 8 rows (N)
    d |= (uint64_t)1 << 46;                          // descriptor version
    return d;                                        // base offset 0, no swizzle
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
                 :: "r"(d), "r"(a), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 :: "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                    "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
                    "r"(v[15]) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                   "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15])
                 : "r"(taddr) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// kernel value without its constant factor (see Green<>). 3D: the PTX
// approximate reciprocal square root with subnormals flushed (rsqrt(+inf) = 0
// gives the masked sources their zero); touching-leaf tiles also zero r^2 <=
// FLT_MIN (pairs closer than 1.1e-19, coincident points included). 2D: log r^2,
// zero for r^2 = +inf (masked) and, on touching-leaf tiles, for r^2 = 0.
template <int KIND, bool ADJ> __device__ __forceinline__ float tc_green(float r2) {
    if (KIND == 0) {
        const bool on = r2 < 3.0e38f && (!ADJ || r2 > 0.f);
        return on ? logf(r2) : 0.f;
    }
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2));
    return (!ADJ || r2 > 1.17549435e-38f) ? y : 0.f;
}

// 16 sources (j0 .. j0+15) against this thread's target, two sources per
// paired FP32 instruction. c: this row's slot copy of these 16 coordinates
// (axes AX floats apart); xl: the stage's lo parts (touching-leaf tiles);
// nt / nl: the negated target coordinates.
template <int KIND, bool ADJ, int AX>
__device__ __forceinline__ void tc_eval16(const float* c, const float4* xl, int j0, float4 nt, float4 nl,
                                          uint32_t* ghi, uint32_t* glo) {
    const float2 ntx = make_float2(nt.x, nt.x), nty = make_float2(nt.y, nt.y), ntz = make_float2(nt.z, nt.z);
    float2 nlx, nly, nlz;
    if (ADJ) nlx = make_float2(nl.x, nl.x), nly = make_float2(nl.y, nl.y), nlz = make_float2(nl.z, nl.z);
    const float2 m1 = make_float2(-1.f, -1.f), split = make_float2(8193.f, 8193.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        // four sources per axis in one 16-byte load
        const float4 X = *reinterpret_cast<const float4*>(&c[4 * q]);
        const float4 Y = *reinterpret_cast<const float4*>(&c[AX + 4 * q]);
        const float4 Z = *reinterpret_cast<const float4*>(&c[2 * AX + 4 * q]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int jj = 4 * q + 2 * h;
            float2 dx = __fadd2_rn(h ? make_float2(X.z, X.w) : make_float2(X.x, X.y), ntx);
            float2 dy = __fadd2_rn(h ? make_float2(Y.z, Y.w) : make_float2(Y.x, Y.y), nty);
            float2 dz = __fadd2_rn(h ? make_float2(Z.z, Z.w) : make_float2(Z.x, Z.y), ntz);
            if (ADJ) {
                const float4 l0 = xl[j0 + jj], l1 = xl[j0 + jj + 1];
                dx = __fadd2_rn(dx, __fadd2_rn(make_float2(l0.x, l1.x), nlx));
                dy = __fadd2_rn(dy, __fadd2_rn(make_float2(l0.y, l1.y), nly));
                dz = __fadd2_rn(dz, __fadd2_rn(make_float2(l0.z, l1.z), nlz));
            }
            float2 r2 = __fmul2_rn(dx, dx);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            const float2 g = make_float2(tc_green<KIND, ADJ>(r2.x), tc_green<KIND, ADJ>(r2.y));
            // Veltkamp's split: hi = t - (t - g) with t = (2^13 + 1) g keeps 11
            // significant bits of g (exactly a TF32 value, rounded to
            // nearest); lo = g - hi is exact
            const float2 t = __fmul2_rn(g, split);
            const float2 hi = __ffma2_rn(__ffma2_rn(g, m1, t), m1, t);
            const float2 lo = __ffma2_rn(hi, m1, g);
            ghi[jj] = __float_as_uint(hi.x);
            ghi[jj + 1] = __float_as_uint(hi.y);
            glo[jj] = __float_as_uint(lo.x);
            glo[jj + 1] = __float_as_uint(lo.y);
        }
    }
}

// One source chunk for right-hand sides r0 .. r0+31, laid out as the stage
// holds it: the B operand in the shared-memory layout of the MMA (element
// (n, j) at float (j/4)*128 + n*4 + j%4), split into TF32 hi (rounded to
// nearest) and lo = q - hi, then the chunk's 32 source coordinates (hi part
// minus the box centre: FP32 then resolves them to the box size, not to the
// domain size) and their lo parts; entries past the chunk and columns past
// nrhs are zero.
// Complex charges (CPLX, the blob of tc_cnear_kernel): B column n < 16 holds
// the real part of right-hand side r0 + n, column 16 + n its imaginary part
// (Q interleaved (re, im)); B' = [-imaginary | real] follows B; then the
// coordinates.
// Thread: n = tid % 32, sources 4 (tid / 32) .. +3.
template <bool CPLX = false>
__global__ void __launch_bounds__(256) tc_bprep_kernel(const int64_t* __restrict__ chunk_start,
                                                       const int32_t* __restrict__ chunk_cnt,
                                                       const float* __restrict__ Q, int nrhs, int r0,
                                                       const float4* __restrict__ X, const float4* __restrict__ Xlo,
                                                       const float4* __restrict__ center, float* __restrict__ B) {
    constexpr int kBlob = CPLX ? 4 * 1024 + 2 * 128 : kChunkFloats;
    constexpr int kXoff = CPLX ? 4096 : 2048;
    const int64_t ch = blockIdx.x;
    const int n = threadIdx.x & 31, jq = threadIdx.x >> 5;
    const int64_t start = chunk_start[ch];
    const int cnt = chunk_cnt[ch];
    const int rr = CPLX ? r0 + (n & 15) : r0 + n;         // the right-hand side of column n
    float v[4], w[4];                                      // B and (CPLX) B' of column n
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int j = 4 * jq + c;
        v[c] = w[c] = 0.f;
        if (j < cnt && rr < nrhs) {
            if constexpr (CPLX) {
                const float2 z = reinterpret_cast<const float2*>(Q)[(start + j) * nrhs + rr];
                v[c] = n < 16 ? z.x : z.y;
                w[c] = n < 16 ? -z.y : z.x;
            } else {
                v[c] = Q[(start + j) * nrhs + rr];
            }
        }
    }
    float* blob = B + ch * kBlob;
#pragma unroll
    for (int part = 0; part < (CPLX ? 2 : 1); ++part) {
        const float* x = part ? w : v;
        float4 h, l;
        h.x = __uint_as_float(to_tf32(x[0]));
        h.y = __uint_as_float(to_tf32(x[1]));
        h.z = __uint_as_float(to_tf32(x[2]));
        h.w = __uint_as_float(to_tf32(x[3]));
        l = make_float4(x[0] - h.x, x[1] - h.y, x[2] - h.z, x[3] - h.w);
        *reinterpret_cast<float4*>(blob + 2048 * part + jq * 128 + n * 4) = h;
        *reinterpret_cast<float4*>(blob + 2048 * part + 1024 + jq * 128 + n * 4) = l;
    }
    // the chunk's coordinates: hi parts measured from the box centre, then
    // the lo parts (zero past cnt)
    if (threadIdx.x < 64) {
        const int j = threadIdx.x & 31;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < cnt) {
            if (threadIdx.x < 32) {
                const float4 x = X[start + j], o = center[ch];
                c = make_float4(x.x - o.x, x.y - o.y, x.z - o.z, 0.f);
            } else {
                c = Xlo[start + j];
            }
        }
        reinterpret_cast<float4*>(blob + kXoff)[threadIdx.x] = c;
    }
}

// Stored-operator mode, per-tile store: a tile's 32 columns come in 8 quads
// of 4 (quad h * 4 + q holds columns 16 h + 4 q .. + 3); the tile keeps the
// quads some row of its item keeps a source in (bit of qmask[tile]), each as
// nrows float4 (unscaled FP32, zero where a row's slot skips the source), so
// that compute thread (row, half) reads its quads as 16-byte words with
// consecutive rows adjacent. Tiles follow each other from A + abase[item].
constexpr int kTileFloats = 128 * 32;          // the largest tile
// float4 index of (row, quad) in a tile with quad mask qm
__device__ __forceinline__ int tile_word(uint32_t qm, int quad, int row, int nrows) {
    return __popc(qm & ((1u << quad) - 1u)) * nrows + row;
}

// REC: the fill pass of a stored-operator mode also writes the kernel values
// it evaluates to a.A: kRecTiles every tile's values as the MMA consumes them
// (hi + lo, masked), kRecSym the blocks this tile records for the symmetric
// store (every source of the chunk, unmasked).
constexpr int kRecNone = 0, kRecTiles = 1, kRecSym = 2;
template <int KIND, int REC = kRecNone, int NS = kNS>
__global__ void __launch_bounds__(kTcThreads, 2) tc_near_kernel(const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcShared<NS>& S = *reinterpret_cast<TcShared<NS>*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const TcItem* itp = a.items + blockIdx.x;
    const int64_t row_off = itp->row_off;
    const int nrows = itp->nrows, nslot = itp->nslot, list_lo = itp->list_lo;
    const int ntile = itp->list_hi - list_lo;

    if (tid == 0) {
        S.slots = 0;
        for (int s = 0; s < NS; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sm_addr(&S.full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(sm_addr(&S.afull[s])), "r"(kTcCompute));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sm_addr(&S.empty[s])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(sm_addr(&S.tmem)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = S.tmem;
    bool err = false;

    if (warp == kTcCompute / 32) {
        // ---------------- producer warp: bulk copies up to NS tiles ahead ----------------
        // the lanes fetch the descriptors of 32 tiles at a time; lane 0
        // issues each tile's copies
        for (int t0 = 0; t0 < ntile; t0 += 32) {
            const int d_chunk = t0 + lane < ntile ? a.tiles[list_lo + t0 + lane].chunk : 0;
            const int nb = min(32, ntile - t0);
            for (int i = 0; i < nb; ++i) {
                const int t = t0 + i;
                const int s = t % NS;
                const int chunk = __shfl_sync(0xffffffffu, d_chunk, i);
                if (t >= NS && !mbar_wait(sm_addr(&S.empty[s]), (uint32_t)(((t - NS) / NS) & 1), a.wait_ns)) err = true;
                const bool hold = t == 0 && (int)blockIdx.x == a.withhold_item;
                if (hold && !withhold_first_tile(sm_addr(&S.afull[0]), a.wait_ns)) err = true;
                if (lane == 0) {
                    // two bulk copies: the chunk (B hi, B lo, coordinates) and
                    // the tile's descriptor
                    const uint32_t bar = sm_addr(&S.full[s]);
                    mbar_arrive_tx(bar, 4u * kChunkFloats + 64u);
                    bulk_g2s_hint(sm_addr(S.st[s].bhi), a.B + (int64_t)chunk * kChunkFloats, 4u * kChunkFloats, bar,
                                  l2_evict_last());
                    bulk_g2s_hint(sm_addr(&S.st[s].tile), a.tiles + list_lo + t, 64u, bar, l2_evict_first());
                    if (hold && !mbar_wait(bar, 0u, a.wait_ns)) err = true;
                }
                __syncwarp();
            }
        }
        if (lane == 0) {
            // all bulk copies have landed before the CTA may exit
            for (int t = (ntile > NS ? ntile - NS : 0); t < ntile; ++t)
                if (!mbar_wait(sm_addr(&S.full[t % NS]), (uint32_t)((t / NS) & 1), a.wait_ns)) err = true;
        }
    } else if (warp == kTcCompute / 32 + 1) {
        // ---------------- MMA issuer (one thread) ----------------
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                                   ((128u >> 4) << 24);
            for (int m = 0; m < ntile; ++m) {
                const int s = m % NS, ab = m % kNA;
                if (!mbar_wait(sm_addr(&S.afull[s]), (uint32_t)((m / NS) & 1), a.wait_ns)) err = true;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t bh = sm_addr(S.st[s].bhi), bl = sm_addr(S.st[s].blo);
                const uint32_t d = tbase + kColD + 32u * (m & 1);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t ahi = tbase + kColA + 64u * ab + 8u * k, alo = ahi + 32u;
                    mma_tf32(d, ahi, smem_desc(bh + 2u * kBLbo * k), idesc, k > 0 ? 1u : 0u);
                    mma_tf32(d, ahi, smem_desc(bl + 2u * kBLbo * k), idesc, 1u);
                    mma_tf32(d, alo, smem_desc(bh + 2u * kBLbo * k), idesc, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(sm_addr(&S.empty[s])) : "memory");
            }
        }
    } else {
        // ---------------- compute warps ----------------
        const int row = tid & 127, half = tid >> 7;
        const bool valid = row < nrows;
        int myslot = 0;
        for (int c = 1; c < nslot; ++c)
            if (row >= itp->slot_start[c]) myslot = c;
        float4 tx = make_float4(0.f, 0.f, 0.f, 0.f), tl = tx;
        if (valid) {
            tx = a.X[row_off + row];
            tl = a.Xlo[row_off + row];
        }
        const float4 nl = make_float4(-tl.x, -tl.y, -tl.z, 0.f);
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        // the slots this warp's 32 rows fall in: s_lo .. s_lo + nsw - 1
        const int r_first = 32 * (warp & 3), r_last = min(r_first + 31, nrows - 1);
        int s_lo = 0, s_hi = 0;
        for (int c = 1; c < nslot; ++c) {
            if (r_first >= itp->slot_start[c]) s_lo = c;
            if (r_last >= itp->slot_start[c]) s_hi = c;
        }
        const int nsw = max(1, s_hi - s_lo + 1);
        const int myloc = min(max(myslot - s_lo, 0), kMaxSlots - 1);
        float* wc = S.wc[warp];
        constexpr int kCols = kTcN / kTpr;                     // accumulator columns this thread owns
        constexpr uint32_t kKeepMask = kSrcPerThread == 32 ? 0xFFFFFFFFu : (1u << kSrcPerThread) - 1u;
        const int j0 = kSrcPerThread * half;
        int64_t tfill = 0;                                     // per-tile fill: floats of the tiles before
        // fill pass: this row's row chunk and its row in it
        int rk = 0, rl = row, rm = 1;
        int64_t rref0 = 0;
        if constexpr (REC == kRecSym) {
            const ItemSym* is = a.isym + blockIdx.x;
            rm = is->m;
            rref0 = is->ref0;
            for (int k = 1; k < rm; ++k)
                if (row >= is->ro[k]) rk = k;
            rl = row - is->ro[rk];
        }
        // two-level FP32 sum: acc adds the tiles of a group of kTcGroup, the
        // shared-memory `outer` adds the groups (keeps long lists accurate)
        float acc[kCols];
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            acc[c] = 0.f;
            S.outer[c][tid] = 0.f;
        }
        auto drain = [&](int m) {                              // add tile m's accumulator
            if (!mbar_wait(sm_addr(&S.empty[m % NS]), (uint32_t)((m / NS) & 1), a.wait_ns)) err = true;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t v[kCols];
            const uint32_t col = tbase + lane_off + kColD + 32u * (m & 1) + (uint32_t)(kCols * half);
            if constexpr (kCols == 32) tmem_ld32(col, v);
            else tmem_ld16(col, v);
#pragma unroll
            for (int c = 0; c < kCols; ++c) acc[c] += __uint_as_float(v[c]);
            if (m % kTcGroup == kTcGroup - 1) {
#pragma unroll
                for (int c = 0; c < kCols; ++c) {
                    S.outer[c][tid] += acc[c];
                    acc[c] = 0.f;
                }
            }
        };
        for (int u = 0; u < ntile; ++u) {
            const int s = u % NS;
            if (!mbar_wait(sm_addr(&S.full[s]), (uint32_t)((u / NS) & 1), a.wait_ns)) err = true;
            TcStage& st = S.st[s];
            const bool adj = (st.tile.flags & TASK_ADJ) != 0;
            // the target measured from the source box's centre (the frame of
            // the chunk's coordinates); touching leaves keep hi and lo apart
            const float cx = st.tile.cen[0], cy = st.tile.cen[1], cz = st.tile.cen[2];
            const float4 nt = adj ? make_float4(cx - tx.x, cy - tx.y, cz - tx.z, 0.f)
                                  : make_float4((cx - tx.x) - tl.x, (cy - tx.y) - tl.y, (cz - tx.z) - tl.z, 0.f);
            const uint32_t keep = valid ? (st.tile.keep[myslot] >> j0) & kKeepMask : 0u;
            // this warp's copy of its sources per slot and axis; a skipped
            // source (and any j >= cnt, never kept) sits at kFar. Every lane
            // has finished reading the previous tile's copy.
            __syncwarp();
            for (int p = lane; p < nsw * kSrcPerThread; p += 32) {
                const int ls = p / kSrcPerThread, jj = p % kSrcPerThread;
                const float4 v = st.xh[j0 + jj];
                // (the fill pass records every source of the chunk, unmasked:
                // each reader of a stored block applies its own keep mask)
                const bool kept = REC == kRecSym ? (j0 + jj < st.tile.cnt)
                                                 : ((st.tile.keep[s_lo + ls] >> (j0 + jj)) & 1u) != 0u;
                float* d = wc + ls * kWarpSlotFloats + jj;
                d[0] = kept ? v.x : kFar;
                d[kSrcPerThread] = kept ? v.y : kFar;
                d[2 * kSrcPerThread] = kept ? v.z : kFar;
            }
            __syncwarp();
            if (u >= 2) drain(u - 2);                          // frees accumulator (u & 1)
            // A buffer u % kNA was last read by MMA(u - kNA), complete since drain(u - 2)
            const uint32_t acol = tbase + lane_off + kColA + 64u * (u % kNA) + (uint32_t)j0;
            const float* c = wc + myloc * kWarpSlotFloats;
            const bool none = REC != kRecSym && __all_sync(0xffffffffu, keep == 0);
#pragma unroll
            for (int g = 0; g < kSrcPerThread / 16; ++g) {
                uint32_t ghi[16], glo[16];
                if (none) {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) ghi[jj] = glo[jj] = 0u;
                } else if (adj) {
                    tc_eval16<KIND, true, kSrcPerThread>(c + 16 * g, st.xl, j0 + 16 * g, nt, nl, ghi, glo);
                } else {
                    tc_eval16<KIND, false, kSrcPerThread>(c + 16 * g, st.xl, j0 + 16 * g, nt, nl, ghi, glo);
                }
                tmem_st16(acol + 16u * g, ghi);
                tmem_st16(acol + 32u + 16u * g, glo);
                if constexpr (REC == kRecTiles) {
                    const uint32_t qm = a.qmask[list_lo + u];
                    float4* dst = reinterpret_cast<float4*>(a.A + a.abase[blockIdx.x] + tfill);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int jj = 4 * q, quad = 4 * half + q;
                        if (valid && ((qm >> quad) & 1u)) dst[tile_word(qm, quad, row, nrows)] =
                            make_float4(__uint_as_float(ghi[jj]) + __uint_as_float(glo[jj]),
                                        __uint_as_float(ghi[jj + 1]) + __uint_as_float(glo[jj + 1]),
                                        __uint_as_float(ghi[jj + 2]) + __uint_as_float(glo[jj + 2]),
                                        __uint_as_float(ghi[jj + 3]) + __uint_as_float(glo[jj + 3]));
                    }
                    tfill += (int64_t)__popc(qm) * nrows * 4;
                }
                if constexpr (REC == kRecSym) {
                    // this row's block of the tile, if this tile records it
                    // (stored as this row chunk x the tile's chunk)
                    const BlockRef rf = a.refs[rref0 + (int64_t)u * rm + rk];
                    if (valid && (rf.flags & kRefRecord)) {
                        const int jb = j0 + 16 * g;
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj)
                            if (jb + jj < st.tile.cnt)
                                a.A[rf.off + (int64_t)(jb + jj) * rf.pitch + rl] =
                                    __uint_as_float(ghi[jj]) + __uint_as_float(glo[jj]);
                    }
                }
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(sm_addr(&S.afull[s]));
        }
        for (int m = (ntile >= 2 ? ntile - 2 : 0); m < ntile; ++m) drain(m);
#pragma unroll
        for (int c = 0; c < kCols; ++c) acc[c] += S.outer[c][tid];
        if (valid) {
            const float scale = (float)green_scale<KIND>();
            const int64_t base = (row_off + row) * a.nrhs;
            const int c0 = a.r0 + kCols * half;
#pragma unroll
            for (int c = 0; c < kCols; ++c)
                if (c0 + c < a.nrhs) a.U[base + c0 + c] = scale * acc[c];
        }
    }
    if (err) atomicExch(a.status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(kTmemCols));
    }
}

// ---------------------------------------------------------------------------
// Stored-operator mode, per-tile store: the same translations with every
// tile's kernel values read from the tiles the fill pass (tc_near_kernel with
// REC = kRecTiles) wrote, instead of evaluated. Tile u of an item with nrows
// rows keeps its nrows x 32 values (unscaled FP32, zero where a row's slot
// skips the source) at A + abase[item] + u * nrows * 32, ordered so that
// compute thread (row, half) reads its 16 values as four 16-byte words with
// consecutive rows adjacent: value (row, j = 16 half + 4 q + e) at
// ((half * 4 + q) * nrows + row) * 4 + e. Per tile the producer copies 24 KB
// at most (the chunk's B hi + lo and the kernel tile); the compute warps only
// split the values into TF32 hi + lo and write A to tensor memory. The MMA
// issue, the accumulator drain and the two-level sum are those of
// tc_near_kernel, so both give the same result bit for bit. Bound: HBM,
// nrows x 128 bytes of kernel values per tile.
static_assert(kSrcPerThread == 16, "stored tiles assume two compute threads per row");
// Four stages in flight need the shared memory that tc_near_kernel gives to
// the outer sums, so here they live in tensor memory, where two A buffers
// leave room: D0, D1 [0, 64), A[b] hi at 64 + 64 b, lo at 96 + 64 b (b < 2),
// the outer sums at [192, 224). Two A buffers suffice: the buffer of tile u
// was last read by MMA(u - 2), which drain(u - 2) has waited for before tile
// u is written.
// NST data stages (24 KB each): 4 with two CTAs per SM, or 8 with one CTA
// per SM (the autotuner times both).
constexpr int kNAS = 2;                        // A buffers
constexpr uint32_t kColOuter = 192;
struct alignas(128) TcTileStage {
    float b[2 * 1024];                         // B hi, B lo (the first 8 KB of the chunk block)
    float4 ga[kTileFloats / 4];                // the tile's kept quads
    uint32_t qm;                               // which quads (written by the producer)
};
template <int NST>
struct TcTileShared {
    TcTileStage st[NST];
    uint64_t full[NST], afull[NST], empty[NST];
    uint32_t tmem;
};
template <int NST>
constexpr int tcs_smem_request() { return NST <= 4 ? 100 * 1024 : 200 * 1024; }
static_assert(sizeof(TcTileShared<4>) <= tcs_smem_request<4>(), "shared memory plan (per-tile store)");
static_assert(sizeof(TcTileShared<8>) <= tcs_smem_request<8>(), "shared memory plan (per-tile store)");

template <int KIND, int NST>
__global__ void __launch_bounds__(kTcThreads, NST <= 4 ? 2 : 1) tc_stored_kernel(const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcTileShared<NST>& S = *reinterpret_cast<TcTileShared<NST>*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const TcItem* itp = a.items + blockIdx.x;
    const int64_t row_off = itp->row_off;
    const int nrows = itp->nrows, list_lo = itp->list_lo;
    const int ntile = itp->list_hi - list_lo;

    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sm_addr(&S.full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(sm_addr(&S.afull[s])), "r"(kTcCompute));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sm_addr(&S.empty[s])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(sm_addr(&S.tmem)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = S.tmem;
    bool err = false;

    if (warp == kTcCompute / 32) {
        // ---------------- producer warp ----------------
        const float* tiles_src = a.A + a.abase[blockIdx.x];
        int64_t toff = 0;                                      // floats of the tiles before
        for (int t0 = 0; t0 < ntile; t0 += 32) {
            const int d_chunk = t0 + lane < ntile ? a.tiles[list_lo + t0 + lane].chunk : 0;
            const uint32_t d_qm = t0 + lane < ntile ? a.qmask[list_lo + t0 + lane] : 0u;
            const int nb = min(32, ntile - t0);
            for (int i = 0; i < nb; ++i) {
                const int t = t0 + i;
                const int s = t % NST;
                const int chunk = __shfl_sync(0xffffffffu, d_chunk, i);
                const uint32_t qm = __shfl_sync(0xffffffffu, d_qm, i);
                const uint32_t tile_bytes = 16u * (uint32_t)__popc(qm) * (uint32_t)nrows;
                if (t >= NST && !mbar_wait(sm_addr(&S.empty[s]), (uint32_t)(((t - NST) / NST) & 1), a.wait_ns))
                    err = true;
                const bool hold = t == 0 && (int)blockIdx.x == a.withhold_item;
                if (hold && !withhold_first_tile(sm_addr(&S.afull[0]), a.wait_ns)) err = true;
                if (lane == 0) {
                    const uint32_t bar = sm_addr(&S.full[s]);
                    S.st[s].qm = qm;
                    mbar_arrive_tx(bar, 4u * 2048u + tile_bytes);
                    bulk_g2s_hint(sm_addr(S.st[s].b), a.B + (int64_t)chunk * kChunkFloats, 4u * 2048u, bar,
                                  l2_evict_last());
                    if (tile_bytes > 0)
                        bulk_g2s_hint(sm_addr(S.st[s].ga), tiles_src + toff, tile_bytes, bar, l2_evict_first());
                    if (hold && !mbar_wait(bar, 0u, a.wait_ns)) err = true;
                }
                toff += (int64_t)__popc(qm) * nrows * 4;
                __syncwarp();
            }
        }
        if (lane == 0) {
            for (int t = (ntile > NST ? ntile - NST : 0); t < ntile; ++t)
                if (!mbar_wait(sm_addr(&S.full[t % NST]), (uint32_t)((t / NST) & 1), a.wait_ns)) err = true;
        }
    } else if (warp == kTcCompute / 32 + 1) {
        // ---------------- MMA issuer (one thread) ----------------
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                                   ((128u >> 4) << 24);
            for (int m = 0; m < ntile; ++m) {
                const int s = m % NST, ab = m % kNAS;
                if (!mbar_wait(sm_addr(&S.afull[s]), (uint32_t)((m / NST) & 1), a.wait_ns)) err = true;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t bh = sm_addr(S.st[s].b), bl = bh + 4u * 1024u;
                const uint32_t d = tbase + kColD + 32u * (m & 1);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t ahi = tbase + kColA + 64u * ab + 8u * k, alo = ahi + 32u;
                    mma_tf32(d, ahi, smem_desc(bh + 2u * kBLbo * k), idesc, k > 0 ? 1u : 0u);
                    mma_tf32(d, ahi, smem_desc(bl + 2u * kBLbo * k), idesc, 1u);
                    mma_tf32(d, alo, smem_desc(bh + 2u * kBLbo * k), idesc, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(sm_addr(&S.empty[s])) : "memory");
            }
        }
    } else {
        // ---------------- compute warps ----------------
        const int row = tid & 127, half = tid >> 7;
        const bool valid = row < nrows;
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        constexpr int kCols = kTcN / kTpr;
        const int j0 = kSrcPerThread * half;
        float acc[kCols];
        const uint32_t ocol = tbase + lane_off + kColOuter + (uint32_t)(kCols * half);
        {
            uint32_t z[kCols];
#pragma unroll
            for (int c = 0; c < kCols; ++c) {
                acc[c] = 0.f;
                z[c] = 0u;
            }
            tmem_st16(ocol, z);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        // the outer sums: this thread's 16 columns of lane `row`
        auto flush = [&]() {
            uint32_t v[kCols];
            tmem_ld16(ocol, v);
#pragma unroll
            for (int c = 0; c < kCols; ++c) {
                v[c] = __float_as_uint(__uint_as_float(v[c]) + acc[c]);
                acc[c] = 0.f;
            }
            tmem_st16(ocol, v);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        };
        auto drain = [&](int m) {
            if (!mbar_wait(sm_addr(&S.empty[m % NST]), (uint32_t)((m / NST) & 1), a.wait_ns)) err = true;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t v[kCols];
            tmem_ld16(tbase + lane_off + kColD + 32u * (m & 1) + (uint32_t)(kCols * half), v);
#pragma unroll
            for (int c = 0; c < kCols; ++c) acc[c] += __uint_as_float(v[c]);
            if (m % kTcGroup == kTcGroup - 1) flush();
        };
        const float2 m1 = make_float2(-1.f, -1.f), split = make_float2(8193.f, 8193.f);
        for (int u = 0; u < ntile; ++u) {
            const int s = u % NST;
            if (!mbar_wait(sm_addr(&S.full[s]), (uint32_t)((u / NST) & 1), a.wait_ns)) err = true;
            uint32_t ghi[16], glo[16];
            // a stale mask after a bounded wait gave up can only pick a quad
            // inside the 16 KB area (at most 8 quads of nrows <= 128 rows)
            const uint32_t qm = S.st[s].qm & 0xFFu;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int quad = 4 * half + q;
                const float4 g4 = (valid && ((qm >> quad) & 1u)) ? S.st[s].ga[tile_word(qm, quad, row, nrows)]
                                                                 : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 g = h ? make_float2(g4.z, g4.w) : make_float2(g4.x, g4.y);
                    const float2 t = __fmul2_rn(g, split);
                    const float2 hi = __ffma2_rn(__ffma2_rn(g, m1, t), m1, t);
                    const float2 lo = __ffma2_rn(hi, m1, g);
                    const int jj = 4 * q + 2 * h;
                    ghi[jj] = __float_as_uint(hi.x);
                    ghi[jj + 1] = __float_as_uint(hi.y);
                    glo[jj] = __float_as_uint(lo.x);
                    glo[jj + 1] = __float_as_uint(lo.y);
                }
            }
            if (u >= 2) drain(u - 2);
            const uint32_t acol = tbase + lane_off + kColA + 64u * (u % kNAS) + (uint32_t)j0;
            tmem_st16(acol, ghi);
            tmem_st16(acol + 32u, glo);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(sm_addr(&S.afull[s]));
        }
        for (int m = (ntile >= 2 ? ntile - 2 : 0); m < ntile; ++m) drain(m);
        {
            uint32_t v[kCols];
            tmem_ld16(ocol, v);
#pragma unroll
            for (int c = 0; c < kCols; ++c) acc[c] += __uint_as_float(v[c]);
        }
        if (valid) {
            const float scale = (float)green_scale<KIND>();
            const int64_t base = (row_off + row) * a.nrhs;
            const int c0 = a.r0 + kCols * half;
#pragma unroll
            for (int c = 0; c < kCols; ++c)
                if (c0 + c < a.nrhs) a.U[base + c0 + c] = scale * acc[c];
        }
    }
    if (err) atomicExch(a.status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(kTmemCols));
    }
}

// ---------------------------------------------------------------------------
// Stored-operator mode, symmetric store: the same translations with the kernel values read
// from the symmetric store instead of evaluated. Per tile the producer copies
// into a stage the chunk's B hi + lo (8 KB), the tile's SrcTile (its keep
// masks) and BlockRefs, and the row chunks' stored blocks, one after the
// other, into a ring of shared memory (a tile's blocks take 6 KB on average
// and at most 18 KB, so a ring holds several times more tiles in flight than
// fixed per-stage areas would). The compute warps find their row chunk's
// block from the ring base the producer recorded and the sizes of the blocks
// before it, read their row's 16 values directly or transposed, apply the
// row's keep mask, split into TF32 hi + lo and write A to tensor memory. The
// MMA issue, the accumulator drain and the two-level sum are those of
// tc_near_kernel. Bound: HBM, 4 bytes per stored value.
static_assert(kSrcPerThread == 16, "stored tiles assume two compute threads per row");
constexpr int kNSY = 6;                        // stages (B operand, descriptors)
constexpr int kRing = 10240;                   // floats of the block ring (40 KB)
static_assert(kSymFloats <= kRing, "a tile's blocks fit the ring");
struct alignas(128) TcSymStage {
    float b[2 * 1024];                         // B hi, B lo (the first 8 KB of the chunk block)
    SrcTile tile;                              // the tile's descriptor (keep masks, source count)
    BlockRef refs[kMaxRc];                     // its row chunks' blocks
    int32_t rbase;                             // ring float of its first block
};
struct TcSymShared {
    TcSymStage st[kNSY];
    float ring[kRing];
    float outer[kTcN / kTpr][kTcCompute];
    uint64_t full[kNSY], afull[kNSY], empty[kNSY];
    uint32_t tmem;
};
constexpr int kTsySmemRequest = 112 * 1024;   // two CTAs per SM
static_assert(sizeof(TcSymShared) <= kTsySmemRequest, "shared memory plan (symmetric store)");

template <int KIND>
__global__ void __launch_bounds__(kTcThreads, 2) tc_sym_kernel(const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSymShared& S = *reinterpret_cast<TcSymShared*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const TcItem* itp = a.items + blockIdx.x;
    const ItemSym* isp = a.isym + blockIdx.x;
    const int64_t row_off = itp->row_off;
    const int nrows = itp->nrows, nslot = itp->nslot, list_lo = itp->list_lo;
    const int ntile = itp->list_hi - list_lo;
    const int m = isp->m;
    const int64_t ref0 = isp->ref0;

    if (tid == 0) {
        for (int s = 0; s < kNSY; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sm_addr(&S.full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(sm_addr(&S.afull[s])), "r"(kTcCompute));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sm_addr(&S.empty[s])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(sm_addr(&S.tmem)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = S.tmem;
    bool err = false;

    if (warp == kTcCompute / 32) {
        // ---------------- producer warp ----------------
        // lane k < m copies row chunk k's block. The descriptors come in
        // batches of per = 32 / m tiles (lane l holds reference l % m of tile
        // t0 + l / m, and the chunk of tile t0 + l), the next batch loading
        // while this one is issued. Ring space is handed out in tile order:
        // a tile's blocks go contiguously at the head (to the start of the
        // ring if they would wrap), after the oldest tiles whose space that
        // needs have been consumed (their "empty" barrier); lane s % kNSY
        // remembers where tile s's blocks start.
        const int per = 32 / m;
        const uint64_t pol_once = l2_evict_first(), pol_keep = l2_evict_last();
        auto fetch = [&](int t0, int64_t& roff, uint32_t& rbytes, int& ch) {
            roff = 0;
            rbytes = 0u;
            if (lane < per * m && t0 + lane / m < ntile) {
                const BlockRef r = a.refs[ref0 + (int64_t)t0 * m + lane];
                roff = r.off;
                rbytes = r.bytes;
            }
            ch = (lane < per && t0 + lane < ntile) ? a.tiles[list_lo + t0 + lane].chunk : 0;
        };
        int64_t c_off, n_off = 0;
        uint32_t c_bytes, n_bytes = 0u;
        int c_ch, n_ch = 0;
        int64_t head = 0, my_start = 0;
        int tail = 0;
        fetch(0, c_off, c_bytes, c_ch);
        for (int t0 = 0; t0 < ntile; t0 += per) {
            if (t0 + per < ntile) fetch(t0 + per, n_off, n_bytes, n_ch);
            const int nb = min(per, ntile - t0);
            for (int i = 0; i < nb; ++i) {
                const int t = t0 + i;
                const int s = t % kNSY;
                const int src = i * m + (lane < m ? lane : 0);
                const int64_t roff = __shfl_sync(0xffffffffu, c_off, src);
                uint32_t rfl = __shfl_sync(0xffffffffu, c_bytes, src) >> 2;     // floats
                if (lane >= m) rfl = 0u;
                const int chunk = __shfl_sync(0xffffffffu, c_ch, i);
                // this lane's block goes pre floats after the tile's first one
                uint32_t incl = rfl;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const uint32_t pre = incl - rfl;
                const uint32_t totf = __shfl_sync(0xffffffffu, incl, 31);
                if (t >= kNSY) {
                    if (!mbar_wait(sm_addr(&S.empty[s]), (uint32_t)(((t - kNSY) / kNSY) & 1), a.wait_ns)) err = true;
                    tail = max(tail, t - kNSY + 1);        // every tile up to t - kNSY is consumed
                }
                int64_t start = head;
                if (start % kRing + totf > (uint32_t)kRing) start += kRing - start % kRing;
                const int64_t end = start + totf;
                while (tail < t && end - __shfl_sync(0xffffffffu, my_start, tail % kNSY) > kRing) {
                    if (!mbar_wait(sm_addr(&S.empty[tail % kNSY]), (uint32_t)((tail / kNSY) & 1), a.wait_ns)) err = true;
                    ++tail;
                }
                head = end;
                if (lane == s) my_start = start;
                const bool hold = t == 0 && (int)blockIdx.x == a.withhold_item;
                if (hold && !withhold_first_tile(sm_addr(&S.afull[0]), a.wait_ns)) err = true;
                const uint32_t bar = sm_addr(&S.full[s]);
                const int rb = (int)(start % kRing);
                if (lane == 0) {
                    S.st[s].rbase = rb;
                    mbar_arrive_tx(bar, 4u * 2048u + 64u + 16u * (uint32_t)m + 4u * totf);
                    bulk_g2s_hint(sm_addr(S.st[s].b), a.B + (int64_t)chunk * kChunkFloats, 4u * 2048u, bar, pol_keep);
                    bulk_g2s_hint(sm_addr(&S.st[s].tile), a.tiles + list_lo + t, 64u, bar, pol_once);
                    bulk_g2s_hint(sm_addr(S.st[s].refs), a.refs + ref0 + (int64_t)t * m, 16u * (uint32_t)m, bar,
                                  pol_once);
                }
                __syncwarp();                          // the byte count is armed before any block lands
                if (rfl > 0)
                    bulk_g2s_hint(sm_addr(S.ring) + 4u * (uint32_t)(rb + pre), a.A + roff, 4u * rfl, bar, pol_once);
                if (hold && lane == 0 && !mbar_wait(bar, 0u, a.wait_ns)) err = true;
                __syncwarp();
            }
            c_off = n_off;
            c_bytes = n_bytes;
            c_ch = n_ch;
        }
        if (lane == 0) {
            for (int t = (ntile > kNSY ? ntile - kNSY : 0); t < ntile; ++t)
                if (!mbar_wait(sm_addr(&S.full[t % kNSY]), (uint32_t)((t / kNSY) & 1), a.wait_ns)) err = true;
        }
    } else if (warp == kTcCompute / 32 + 1) {
        // ---------------- MMA issuer (one thread) ----------------
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                                   ((128u >> 4) << 24);
            for (int mm = 0; mm < ntile; ++mm) {
                const int s = mm % kNSY, ab = mm % kNA;
                if (!mbar_wait(sm_addr(&S.afull[s]), (uint32_t)((mm / kNSY) & 1), a.wait_ns)) err = true;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t bh = sm_addr(S.st[s].b), bl = bh + 4u * 1024u;
                const uint32_t d = tbase + kColD + 32u * (mm & 1);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t ahi = tbase + kColA + 64u * ab + 8u * k, alo = ahi + 32u;
                    mma_tf32(d, ahi, smem_desc(bh + 2u * kBLbo * k), idesc, k > 0 ? 1u : 0u);
                    mma_tf32(d, ahi, smem_desc(bl + 2u * kBLbo * k), idesc, 1u);
                    mma_tf32(d, alo, smem_desc(bh + 2u * kBLbo * k), idesc, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(sm_addr(&S.empty[s])) : "memory");
            }
        }
    } else {
        // ---------------- compute warps ----------------
        const int row = tid & 127, half = tid >> 7;
        const bool valid = row < nrows;
        int myslot = 0;
        for (int c = 1; c < nslot; ++c)
            if (row >= itp->slot_start[c]) myslot = c;
        // this row's row chunk k and its row rl in it
        int rk = 0;
        for (int k = 1; k < m; ++k)
            if (row >= isp->ro[k]) rk = k;
        const int rl = row - isp->ro[rk];
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        constexpr int kCols = kTcN / kTpr;
        const int j0 = kSrcPerThread * half;
        float acc[kCols];
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            acc[c] = 0.f;
            S.outer[c][tid] = 0.f;
        }
        auto drain = [&](int mm) {
            if (!mbar_wait(sm_addr(&S.empty[mm % kNSY]), (uint32_t)((mm / kNSY) & 1), a.wait_ns)) err = true;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t v[kCols];
            tmem_ld16(tbase + lane_off + kColD + 32u * (mm & 1) + (uint32_t)(kCols * half), v);
#pragma unroll
            for (int c = 0; c < kCols; ++c) acc[c] += __uint_as_float(v[c]);
            if (mm % kTcGroup == kTcGroup - 1) {
#pragma unroll
                for (int c = 0; c < kCols; ++c) {
                    S.outer[c][tid] += acc[c];
                    acc[c] = 0.f;
                }
            }
        };
        const float2 m1 = make_float2(-1.f, -1.f), split = make_float2(8193.f, 8193.f);
        for (int u = 0; u < ntile; ++u) {
            const int s = u % kNSY;
            const bool landed = mbar_wait(sm_addr(&S.full[s]), (uint32_t)((u / kNSY) & 1), a.wait_ns);
            if (!landed) err = true;
            const TcSymStage& st = S.st[s];
            // the row's kept sources of this tile, and where its block sits
            uint32_t keep = valid ? (st.tile.keep[myslot] >> j0) & 0xFFFFu : 0u;
            // this row chunk's block: after the tile's earlier blocks in the ring
            int boff = st.rbase;
            for (int k = 0; k < rk; ++k) boff += (int)(st.refs[k].bytes >> 2);
            const BlockRef rf = st.refs[rk];
            const bool tr = (rf.flags & kRefTransposed) != 0;
            const int P = rf.pitch;
            // only a stage whose copies landed is read, and only inside its
            // block (a stored pitch is at most 33, a block lies in the ring):
            // after a bounded wait gave up the descriptors may be stale, and
            // the row then contributes zeros
            if (!landed || P > 33 || boff < 0 || boff + (int)(rf.bytes >> 2) > kRing) keep = 0u;
            // direct: (rl, j) at j P + rl; transposed: at rl P + j
            const float* blk = S.ring + boff + (tr ? rl * P : rl);
            const int step = tr ? 1 : P;
            float gv[16];
            if (__all_sync(0xffffffffu, keep == 0u)) {
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) gv[jj] = 0.f;
            } else {
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) gv[jj] = ((keep >> jj) & 1u) ? blk[(j0 + jj) * step] : 0.f;
            }
            uint32_t ghi[16], glo[16];
#pragma unroll
            for (int jj = 0; jj < 16; jj += 2) {
                const float2 g = make_float2(gv[jj], gv[jj + 1]);
                const float2 t = __fmul2_rn(g, split);
                const float2 hi = __ffma2_rn(__ffma2_rn(g, m1, t), m1, t);
                const float2 lo = __ffma2_rn(hi, m1, g);
                ghi[jj] = __float_as_uint(hi.x);
                ghi[jj + 1] = __float_as_uint(hi.y);
                glo[jj] = __float_as_uint(lo.x);
                glo[jj + 1] = __float_as_uint(lo.y);
            }
            if (u >= 2) drain(u - 2);
            const uint32_t acol = tbase + lane_off + kColA + 64u * (u % kNA) + (uint32_t)j0;
            tmem_st16(acol, ghi);
            tmem_st16(acol + 32u, glo);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(sm_addr(&S.afull[s]));
        }
        for (int mm = (ntile >= 2 ? ntile - 2 : 0); mm < ntile; ++mm) drain(mm);
#pragma unroll
        for (int c = 0; c < kCols; ++c) acc[c] += S.outer[c][tid];
        if (valid) {
            const float scale = (float)green_scale<KIND>();
            const int64_t base = (row_off + row) * a.nrhs;
            const int c0 = a.r0 + kCols * half;
#pragma unroll
            for (int c = 0; c < kCols; ++c)
                if (c0 + c < a.nrhs) a.U[base + c0 + c] = scale * acc[c];
        }
    }
    if (err) atomicExch(a.status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(kTmemCols));
    }
}

}  // namespace skel
