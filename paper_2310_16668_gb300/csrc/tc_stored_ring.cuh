// Per-tile store, split rings: the arithmetic of tc_stored_kernel (the same
// tiles, split, MMAs, drains and sums, so the same bits), with the tile's
// kernel values and its B operand in two separate rings of shared memory.
// The values (up to 16 KB a tile) are only read by the compute warps, which
// release their slot as soon as their quads are in registers; the B operand
// (8 KB) is read by the MMAs and released by their commit. In tc_stored_kernel
// one stage holds both until the MMAs finish, so the values of the next tiles
// wait behind the tensor core; here their slots turn over a tile earlier and
// NA value slots + NB operand slots fit where four whole stages did.
// Bound: HBM, as tc_stored_kernel.
#pragma once

#include "tc_kernels.cuh"

namespace skel {

struct alignas(128) TcValSlot {
    float4 ga[kTileFloats / 4];                // the tile's kept quads
    uint32_t qm;                               // which quads (written by the producer)
};
struct alignas(128) TcBSlot {
    float b[2 * 1024];                         // B hi, B lo
};
template <int NA, int NB>
struct TcRingShared {
    TcValSlot va[NA];
    TcBSlot bb[NB];
    uint64_t fullA[NA], emptyA[NA], afull[NA];
    uint64_t fullB[NB], emptyB[NB];
    uint32_t tmem;
};
template <int NA, int NB>
constexpr int tcr_smem_request() { return (int)sizeof(TcRingShared<NA, NB>) + 128; }
static_assert(tcr_smem_request<5, 3>() <= 113 * 1024, "two CTAs per SM");

template <int KIND, int NA, int NB>
__global__ void __launch_bounds__(kTcThreads, 2) tc_stored_ring_kernel(const TcArgs a) {
    static_assert(NB >= 3, "a drain two tiles back must find its commit phase current");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcRingShared<NA, NB>& S = *reinterpret_cast<TcRingShared<NA, NB>*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const TcItem* itp = a.items + blockIdx.x;
    const int64_t row_off = itp->row_off;
    const int nrows = itp->nrows, list_lo = itp->list_lo;
    const int ntile = itp->list_hi - list_lo;

    if (tid == 0) {
        for (int s = 0; s < NA; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sm_addr(&S.fullA[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(sm_addr(&S.emptyA[s])), "r"(kTcCompute));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(sm_addr(&S.afull[s])), "r"(kTcCompute));
        }
        for (int s = 0; s < NB; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sm_addr(&S.fullB[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sm_addr(&S.emptyB[s])));
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
        // ---------------- producer warp: values NA tiles ahead, B NB tiles ahead ----------------
        const float* tiles_src = a.A + a.abase[blockIdx.x];
        int64_t toff = 0;
        for (int t0 = 0; t0 < ntile; t0 += 32) {
            const int d_chunk = t0 + lane < ntile ? a.tiles[list_lo + t0 + lane].chunk : 0;
            const uint32_t d_qm = t0 + lane < ntile ? a.qmask[list_lo + t0 + lane] : 0u;
            const int nb = min(32, ntile - t0);
            for (int i = 0; i < nb; ++i) {
                const int t = t0 + i;
                const int sa = t % NA, sb = t % NB;
                const int chunk = __shfl_sync(0xffffffffu, d_chunk, i);
                const uint32_t qm = __shfl_sync(0xffffffffu, d_qm, i);
                const uint32_t tile_bytes = 16u * (uint32_t)__popc(qm) * (uint32_t)nrows;
                // the values: their slot is free once the compute warps read tile t - NA
                if (t >= NA && !mbar_wait(sm_addr(&S.emptyA[sa]), (uint32_t)(((t - NA) / NA) & 1), a.wait_ns))
                    err = true;
                const bool hold = t == 0 && (int)blockIdx.x == a.withhold_item;
                if (hold && !withhold_first_tile(sm_addr(&S.afull[0]), a.wait_ns)) err = true;
                if (lane == 0) {
                    const uint32_t bar = sm_addr(&S.fullA[sa]);
                    S.va[sa].qm = qm;
                    mbar_arrive_tx(bar, tile_bytes);
                    if (tile_bytes > 0)
                        bulk_g2s_hint(sm_addr(S.va[sa].ga), tiles_src + toff, tile_bytes, bar, l2_evict_first());
                    if (hold && !mbar_wait(bar, 0u, a.wait_ns)) err = true;
                }
                toff += (int64_t)__popc(qm) * nrows * 4;
                // the B operand: its slot is free once MMA(t - NB) has finished
                if (t >= NB && !mbar_wait(sm_addr(&S.emptyB[sb]), (uint32_t)(((t - NB) / NB) & 1), a.wait_ns))
                    err = true;
                if (lane == 0) {
                    const uint32_t bar = sm_addr(&S.fullB[sb]);
                    mbar_arrive_tx(bar, 4u * 2048u);
                    bulk_g2s_hint(sm_addr(S.bb[sb].b), a.B + (int64_t)chunk * kChunkFloats, 4u * 2048u, bar,
                                  l2_evict_last());
                }
                __syncwarp();
            }
        }
        if (lane == 0) {
            for (int t = (ntile > NA ? ntile - NA : 0); t < ntile; ++t)
                if (!mbar_wait(sm_addr(&S.fullA[t % NA]), (uint32_t)((t / NA) & 1), a.wait_ns)) err = true;
            for (int t = (ntile > NB ? ntile - NB : 0); t < ntile; ++t)
                if (!mbar_wait(sm_addr(&S.fullB[t % NB]), (uint32_t)((t / NB) & 1), a.wait_ns)) err = true;
        }
    } else if (warp == kTcCompute / 32 + 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                                   ((128u >> 4) << 24);
            for (int m = 0; m < ntile; ++m) {
                const int sa = m % NA, sb = m % NB, ab = m % kNAS;
                if (!mbar_wait(sm_addr(&S.afull[sa]), (uint32_t)((m / NA) & 1), a.wait_ns)) err = true;
                if (!mbar_wait(sm_addr(&S.fullB[sb]), (uint32_t)((m / NB) & 1), a.wait_ns)) err = true;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t bh = sm_addr(S.bb[sb].b), bl = bh + 4u * 1024u;
                const uint32_t d = tbase + kColD + 32u * (m & 1);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t ahi = tbase + kColA + 64u * ab + 8u * k, alo = ahi + 32u;
                    mma_tf32(d, ahi, smem_desc(bh + 2u * kBLbo * k), idesc, k > 0 ? 1u : 0u);
                    mma_tf32(d, ahi, smem_desc(bl + 2u * kBLbo * k), idesc, 1u);
                    mma_tf32(d, alo, smem_desc(bh + 2u * kBLbo * k), idesc, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(sm_addr(&S.emptyB[sb])) : "memory");
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
        // tile m's MMAs are done once its B slot's commit phase has completed
        auto drain = [&](int m) {
            if (!mbar_wait(sm_addr(&S.emptyB[m % NB]), (uint32_t)((m / NB) & 1), a.wait_ns)) err = true;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t v[kCols];
            tmem_ld16(tbase + lane_off + kColD + 32u * (m & 1) + (uint32_t)(kCols * half), v);
#pragma unroll
            for (int c = 0; c < kCols; ++c) acc[c] += __uint_as_float(v[c]);
            if (m % kTcGroup == kTcGroup - 1) flush();
        };
        const float2 m1 = make_float2(-1.f, -1.f), split = make_float2(8193.f, 8193.f);
        for (int u = 0; u < ntile; ++u) {
            const int sa = u % NA;
            if (!mbar_wait(sm_addr(&S.fullA[sa]), (uint32_t)((u / NA) & 1), a.wait_ns)) err = true;
            const uint32_t qm = S.va[sa].qm & 0xFFu;
            float4 g4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int quad = 4 * half + q;
                g4[q] = (valid && ((qm >> quad) & 1u)) ? S.va[sa].ga[tile_word(qm, quad, row, nrows)]
                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            // the values are in registers: their slot may be refilled
            mbar_arrive(sm_addr(&S.emptyA[sa]));
            uint32_t ghi[16], glo[16];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 g = h ? make_float2(g4[q].z, g4[q].w) : make_float2(g4[q].x, g4[q].y);
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
            mbar_arrive(sm_addr(&S.afull[sa]));
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

}  // namespace skel
