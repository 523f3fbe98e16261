// Tensor-core translations for many right-hand sides (FP32_TC precision).
//
// For a tile of 128 target rows of one box, the translations are
// U[128 x 32] += G[128 x K] Q[K x 32] over all source entries K of the box's
// tasks, G_ij = G(x_i, y_j) evaluated on the fly. Per tile of 32 sources:
//   * 256 threads evaluate the 128 x 32 kernel block on the CUDA cores (two
//     threads per row, 16 sources each), split every value into TF32 hi + lo
//     parts and write them into tensor memory with tcgen05.st (A operand:
//     TMEM lane = target row, column = source);
//   * the 32 x 32 charge block is split the same way into shared memory in
//     the K-major, no-swizzle core-matrix layout (8 rows x 16 bytes; 128 bytes
//     between core matrices along K, 1024 bytes between groups of 8
//     right-hand sides) — the B operand;
//   * one thread issues 12 tcgen05.mma (kind::tf32, M=128, N=32, K=8):
//     hi*hi + hi*lo + lo*hi for each of the 4 K-steps, accumulating in an
//     FP32 tensor-memory tile, and commits them to the tile buffer's mbarrier.
// Two buffers let the kernel evaluation of tile t+1 run while the tensor
// core multiplies tile t. The dropped lo*lo term and the TF32 rounding of the
// lo parts are below 2^-21 of each product. The tensor-memory accumulator
// only ever sums `drain` tiles: two accumulators alternate, and each finished
// one is added into FP32 registers (round to nearest) while the other fills,
// so no long accumulation chain runs inside the tensor core.
//
// Masks: a source slot that a target slot must skip (the regrouped
// subtractions of Algorithm 2) gives G = 0 for those rows. Every wait is
// bounded; on timeout the kernel raises the status word, waits (bounded) for
// its issued MMAs and always frees its tensor memory.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "host.h"
#include "skel_kernels.cuh"

namespace skel {

constexpr int kTcThreads = 256;
constexpr int kTcN = 32;                       // right-hand sides per pass (MMA N)
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kColD = 0, kColA = 64;      // D0 [0,32), D1 [32,64); A_hi[b] at 64+64b, A_lo[b] at 96+64b
constexpr int kSmB = 0;                        // B_hi[2][1024] floats, then B_lo[2][1024]
constexpr int kSmSrc = 16384;                  // src hi [2][32] float4, then lo [2][32]
constexpr int kSmBar = 18432;                  // mbar[2]
constexpr int kSmTmem = 18448;
constexpr int kSmSlots = 18452;
constexpr int kSmTiles = 18464;                // the item's SrcTile descriptors (<= kTcMaxTiles)
constexpr int kTcSmemRequest = 100 * 1024;     // at most two CTAs (2 x 256 TMEM columns) per SM
constexpr int kSpinLimit = 1 << 20;

struct TcArgs {
    const TcItem* items;
    const SrcTile* tiles;
    const int64_t* box_off;
    const int32_t* box_n;
    const int32_t* box_nslot;
    const int32_t* slot_start;
    const float4* X;
    const float4* Xlo;
    const float* Q;
    float* partial;
    int nrhs;
    int r0;                                    // first right-hand side of this pass
    int drain;                                 // tiles accumulated in tensor memory before a drain
    int* status;
};

__device__ __forceinline__ uint32_t sm_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < kSpinLimit; ++it) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((128 >> 4) & 0x3FFF) << 16;     // LBO: next core matrix along K
    d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;    // SBO: next group of 8 rows (N)
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

// kernel value without its constant factor (see Green<>)
template <int KIND> __device__ __forceinline__ float tc_green(float r2) {
    return KIND == 0 ? logf(r2) : rsqrtf(r2);
}

template <int KIND, bool ADJ>
__device__ __forceinline__ void tc_eval16(const float4* sh, const float4* sl, float4 tx, float4 tl, uint32_t keep,
                                          uint32_t* ghi, uint32_t* glo) {
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
        const float4 s = sh[jj];
        float dx = tx.x - s.x, dy = tx.y - s.y, dz = tx.z - s.z;
        if (ADJ) {
            const float4 l = sl[jj];
            dx += tl.x - l.x;
            dy += tl.y - l.y;
            dz += tl.z - l.z;
        }
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        float g = tc_green<KIND>(r2);
        const bool on = ((keep >> jj) & 1u) && (!ADJ || r2 > 0.f);
        g = on ? g : 0.f;
        const uint32_t h = to_tf32(g);
        ghi[jj] = h;
        glo[jj] = to_tf32(g - __uint_as_float(h));
    }
}

template <int KIND>
__global__ void __launch_bounds__(kTcThreads, 2) tc_near_kernel(const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    float* bhi = reinterpret_cast<float*>(sm + kSmB);
    float* blo = bhi + 2 * 1024;
    float4* shi = reinterpret_cast<float4*>(sm + kSmSrc);
    float4* slo = shi + 2 * 32;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kSmBar);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kSmTmem);
    uint32_t* islots = reinterpret_cast<uint32_t*>(sm + kSmSlots);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & 127, half = tid >> 7;
    const TcItem it = a.items[blockIdx.x];
    const int64_t B = it.box;
    const int64_t boff = a.box_off[B];
    const int nB = a.box_n[B];
    const int t = it.r0 + row;
    const bool valid = t < nB;
    const int32_t* ssB = a.slot_start + B * (kMaxSlots + 1);
    int myslot = 0;
    for (int c = 1; c < a.box_nslot[B]; ++c)
        if (t >= ssB[c]) myslot = c;
    float4 tx = make_float4(0.f, 0.f, 0.f, 0.f), tl = tx;
    if (valid) {
        tx = a.X[boff + t];
        tl = a.Xlo[boff + t];
    }
    if (tid == 0) {
        *islots = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sm_addr(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sm_addr(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(sm_addr(tmem_slot)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (valid && half == 0) atomicOr(islots, 1u << myslot);
    __syncthreads();
    const uint32_t item_slots = *islots;
    const uint32_t tbase = *tmem_slot;
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((128u >> 4) << 24);

    float acc[kTcN];
#pragma unroll
    for (int c = 0; c < kTcN; ++c) acc[c] = 0.f;
    int drained = 0;                               // segments already added into acc
    // add the finished accumulator of segment `seg` into acc (warps 0-3)
    auto drain_seg = [&](int seg) {
        if (half == 0) {
            uint32_t v[kTcN];
            tmem_ld32(tbase + lane_off + kColD + 32u * (seg & 1), v);
#pragma unroll
            for (int c = 0; c < kTcN; ++c) acc[c] += __uint_as_float(v[c]);
        }
    };
    // the item's tile descriptors -> shared memory (one coalesced pass)
    SrcTile* stiles = reinterpret_cast<SrcTile*>(sm + kSmTiles);
    const int ntiles = it.tile_hi - it.tile_lo;
    {
        const int4* src = reinterpret_cast<const int4*>(a.tiles + it.tile_lo);
        int4* dst = reinterpret_cast<int4*>(stiles);
        for (int e = tid; e < ntiles * 2; e += kTcThreads) dst[e] = src[e];
    }
    __syncthreads();
    auto needed = [&](int k) {
        const SrcTile& st = stiles[k];
        uint32_t need = 0;
        for (int s = 0; s < st.nseg; ++s) need |= (~(uint32_t)st.seg_mask[s]) & item_slots;
        return need != 0;
    };
    auto next_needed = [&](int k) {
        while (k < ntiles && !needed(k)) ++k;
        return k;
    };
    // register prefetch of one tile: coordinates (threads 0..31) and 4 charges per thread
    const int pj = tid >> 3, pc0 = (tid & 7) * 4;
    const bool vec4 = (a.nrhs & 3) == 0;
    auto prefetch = [&](int k, float4& ph, float4& pl, float* pq) {
        if (k >= ntiles) return;
        const SrcTile& st = stiles[k];
        if (tid < 32) {
            ph = make_float4(0.f, 0.f, 0.f, 0.f);
            pl = ph;
            if (tid < st.cnt) {
                ph = a.X[st.start + tid];
                if (st.flags & TASK_ADJ) pl = a.Xlo[st.start + tid];
            }
        }
        const int rr = a.r0 + pc0;
        const int64_t base = (st.start + pj) * a.nrhs + rr;
        if (pj < st.cnt && vec4 && rr + 3 < a.nrhs) {
            const float4 v = *reinterpret_cast<const float4*>(a.Q + base);
            pq[0] = v.x; pq[1] = v.y; pq[2] = v.z; pq[3] = v.w;
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) pq[c] = (pj < st.cnt && rr + c < a.nrhs) ? a.Q[base + c] : 0.f;
        }
    };
    float4 nh = make_float4(0.f, 0.f, 0.f, 0.f), nl = nh;
    float nq[4] = {0.f, 0.f, 0.f, 0.f};
    int cur = next_needed(0);
    prefetch(cur, nh, nl, nq);

    int n_issued = 0;
    bool ok = true;
    while (cur < ntiles) {
        const SrcTile st = stiles[cur];
        const float4 ch = nh, cl = nl;
        float cq[4] = {nq[0], nq[1], nq[2], nq[3]};
        const int nxt = next_needed(cur + 1);
        prefetch(nxt, nh, nl, nq);
        const int buf = n_issued & 1, use = n_issued >> 1;
        if (use >= 1) {
            const bool w = mbar_wait(sm_addr(&mbar[buf]), (uint32_t)((use - 1) & 1));
            if (!__syncthreads_and(w)) { ok = false; break; }
            // tile n_issued - 2 is complete: if it closed a segment, drain it
            const int done_tile = n_issued - 2;
            if ((done_tile + 1) % a.drain == 0 && done_tile / a.drain == drained) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                drain_seg(drained);
                ++drained;
            }
        }
        const bool adj = (st.flags & TASK_ADJ) != 0;
        // stage source coordinates and the split charge block
        if (tid < 32) {
            shi[buf * 32 + tid] = ch;
            slo[buf * 32 + tid] = cl;
        }
        {
            float* bh = bhi + buf * 1024;
            float* bl = blo + buf * 1024;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int n = pc0 + c;
                const uint32_t h = to_tf32(cq[c]);
                const int w = ((n >> 3) * 1024 + (pj >> 2) * 128 + (n & 7) * 16 + (pj & 3) * 4) >> 2;
                bh[w] = __uint_as_float(h);
                bl[w] = __uint_as_float(to_tf32(cq[c] - __uint_as_float(h)));
            }
        }
        __syncthreads();
        // this thread's 16 sources: which ones its row keeps
        uint32_t keep = 0;
        {
            int sb = 0;
            for (int s = 0; s < st.nseg; ++s) {
                const int e = st.seg_end[s];
                if (!((st.seg_mask[s] >> myslot) & 1))
                    keep |= (uint32_t)(((1ull << e) - 1ull) ^ ((1ull << sb) - 1ull));
                sb = e;
            }
            keep = valid ? (keep >> (16 * half)) & 0xFFFFu : 0u;
        }
        uint32_t ghi[16], glo[16];
        if (__all_sync(0xffffffffu, keep == 0)) {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) ghi[jj] = glo[jj] = 0u;
        } else if (adj) {
            tc_eval16<KIND, true>(shi + buf * 32 + 16 * half, slo + buf * 32 + 16 * half, tx, tl, keep, ghi, glo);
        } else {
            tc_eval16<KIND, false>(shi + buf * 32 + 16 * half, slo + buf * 32 + 16 * half, tx, tl, keep, ghi, glo);
        }
        const uint32_t acol = tbase + lane_off + kColA + 64u * buf + 16u * half;
        tmem_st16(acol, ghi);
        tmem_st16(acol + 32u, glo);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t bh = sm_addr(bhi + buf * 1024), bl = sm_addr(blo + buf * 1024);
            const int seg = n_issued / a.drain;
            const uint32_t d = tbase + kColD + 32u * (seg & 1);
            const bool first = (n_issued % a.drain) == 0;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const uint32_t ahi = tbase + kColA + 64u * buf + 8u * s, alo = ahi + 32u;
                mma_tf32(d, ahi, smem_desc(bh + 256u * s), idesc, (!first || s > 0) ? 1u : 0u);
                mma_tf32(d, ahi, smem_desc(bl + 256u * s), idesc, 1u);
                mma_tf32(d, alo, smem_desc(bh + 256u * s), idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(sm_addr(&mbar[buf])) : "memory");
        }
        ++n_issued;
        cur = nxt;
    }
    if (n_issued > 0) {
        const int last = n_issued - 1;
        const bool w = mbar_wait(sm_addr(&mbar[last & 1]), (uint32_t)((last >> 1) & 1));
        const bool all = __syncthreads_and(w);
        if (all && ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int nseg = last / a.drain + 1;
            for (; drained < nseg; ++drained) drain_seg(drained);
        } else {
            ok = false;
            if (!all) mbar_wait(sm_addr(&mbar[last & 1]), (uint32_t)((last >> 1) & 1));
        }
    }
    if (!ok && tid == 0) atomicExch(a.status, 1);
    if (half == 0 && valid && ok) {
        const float scale = (float)green_scale<KIND>();
        const int64_t base = ((int64_t)(it.slot + (row >> 5)) * kChunk + (row & 31)) * a.nrhs;
#pragma unroll
        for (int c = 0; c < kTcN; ++c)
            if (a.r0 + c < a.nrhs) a.partial[base + a.r0 + c] = scale * acc[c];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(kTmemCols));
    }
}

}  // namespace skel
