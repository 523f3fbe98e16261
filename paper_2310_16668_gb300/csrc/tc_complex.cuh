// Tensor-core translations for the complex 3D Helmholtz kernel (FP32_TC,
// complex64): the building blocks of tc_kernels.cuh (bulk-copy stages,
// mbarrier protocol with bounded waits, TMEM accumulators, 3-pass TF32 split)
// applied to e^{i kappa r} / (4 pi r), with the sine and cosine evaluated on
// the FP32 pipe.
#pragma once

#include "tc_kernels.cuh"

namespace skel {

// ---------------------------------------------------------------------------
// 3D Helmholtz (complex64) on the tensor cores: u = G q with G = G_r + i G_i
// and q = q_r + i q_i is u_r = G_r q_r - G_i q_i, u_i = G_r q_i + G_i q_r, so
// one real accumulator of 32 columns holds [u_r | u_i] of 16 right-hand sides
// as G_r B + G_i B' with B = [q_r | q_i] and B' = [-q_i | q_r]
// (tc_bprep_kernel<true> writes both, TF32 hi + lo). Per tile the MMA issuer
// adds 12 MMAs of G_r (hi, lo) against B and 12 of G_i against B'. Tensor
// memory: the accumulators of two tiles (64 columns) and three A buffers of
// G_r hi, G_r lo, G_i hi, G_i lo (3 x 128 columns): 512 columns, one CTA per
// SM, so the CTA brings its own latency hiding: 4 compute threads per row
// (16 compute warps), 8 sources of a tile each.
constexpr int kTcNc = 16;                      // complex right-hand sides per pass
constexpr uint32_t kTmemColsC = 512;
constexpr uint32_t kColAc = 64;                // A[b]: G_r hi, G_r lo, G_i hi, G_i lo at 64 + 128 b (+0/32/64/96)
constexpr int kChunkFloatsC = 4 * 1024 + 2 * 128;
constexpr int kTprC = 4;                       // compute threads per target row
constexpr int kComputeC = 128 * kTprC;         // compute threads
constexpr int kSrcC = 32 / kTprC;              // sources of a tile per compute thread
constexpr int kColsC = kTcN / kTprC;           // accumulator columns per compute thread
constexpr int kThreadsC = kComputeC + 64;      // + the producer warp and the MMA warp
constexpr int kSlotFloatsC = 3 * kSrcC;
struct alignas(128) TcStageC {
    float bhi[32 * 32];                        // B = [q_r | q_i], TF32 hi
    float blo[32 * 32];                        //   lo
    float bphi[32 * 32];                       // B' = [-q_i | q_r], TF32 hi
    float bplo[32 * 32];                       //   lo
    float4 xh[32];                             // source coordinates (hi)
    float4 xl[32];                             // lo parts (touching-leaf tiles)
    SrcTile tile;                              // the tile's descriptor (its own copy)
};
static_assert(offsetof(TcStageC, tile) == kChunkFloatsC * 4, "chunk blob is contiguous in the stage");
constexpr int kNSC = 6;                        // data stages
template <int NS>
struct TcSharedC {
    TcStageC st[NS];
    float wc[kComputeC / 32][kMaxSlots * kSlotFloatsC];
    float outer[kColsC][kComputeC];
    uint64_t full[NS], afull[NS], empty[NS];
    uint32_t tmem;
};
constexpr int kTccSmemRequest = 144 * 1024;   // one CTA per SM (512 TMEM columns)
static_assert(sizeof(TcSharedC<kNSC>) <= kTccSmemRequest, "shared memory plan");

__device__ __forceinline__ float2 tc_f2(float x) { return make_float2(x, x); }

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 :: "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                    "r"(v[7]) : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// sin and cos of two non-negative arguments x below 2^21: x = n pi/2 + y with
// |y| <= pi/4. n is rounded to nearest by adding 1.5 * 2^23 (the sum's low
// mantissa bits are then n, so n mod 4 is read from its bits: no conversion
// instruction); Cody and Waite's reduction with pi/2 as a sum of three floats,
// the first with 8 significant bits so that n C1 is exact; the Taylor series
// of sin y to the y^9 term and of cos y to the y^10 term (truncation error
// below 2e-9 on |y| <= pi/4); then the quadrant n mod 4 maps (sin, cos) to
// (sin, cos), (cos, -sin), (-sin, -cos), (-cos, sin), the signs as bit flips.
// FP32 pipe and integer logic only, two arguments per paired instruction.
__device__ __forceinline__ void tc_sincos2(float2 x, float2& s, float2& c) {
    constexpr double kHalfPi = 1.57079632679489661923132169163975;
    constexpr float kC1 = 1.5703125f;
    constexpr float kC2 = (float)(kHalfPi - 1.5703125);
    constexpr float kC3 = (float)(kHalfPi - 1.5703125 - (double)kC2);
    constexpr float kTwoOverPi = (float)(1.0 / kHalfPi);
    constexpr float kRound = 12582912.0f;      // 1.5 * 2^23
    const float2 t = __ffma2_rn(x, tc_f2(kTwoOverPi), tc_f2(kRound));
    const float2 mn = __ffma2_rn(t, tc_f2(-1.f), tc_f2(kRound));   // -n (exact)
    float2 y = __ffma2_rn(mn, tc_f2(kC1), x);
    y = __ffma2_rn(mn, tc_f2(kC2), y);
    y = __ffma2_rn(mn, tc_f2(kC3), y);
    const float2 z = __fmul2_rn(y, y);
    float2 ps = __ffma2_rn(z, tc_f2((float)(1.0 / 362880.0)), tc_f2((float)(-1.0 / 5040.0)));
    ps = __ffma2_rn(z, ps, tc_f2((float)(1.0 / 120.0)));
    ps = __ffma2_rn(z, ps, tc_f2((float)(-1.0 / 6.0)));
    const float2 sy = __ffma2_rn(__fmul2_rn(y, z), ps, y);
    float2 pc = __ffma2_rn(z, tc_f2((float)(-1.0 / 3628800.0)), tc_f2((float)(1.0 / 40320.0)));
    pc = __ffma2_rn(z, pc, tc_f2((float)(-1.0 / 720.0)));
    pc = __ffma2_rn(z, pc, tc_f2((float)(1.0 / 24.0)));
    pc = __ffma2_rn(z, pc, tc_f2(-0.5f));
    const float2 cy = __ffma2_rn(z, pc, tc_f2(1.0f));
    const uint32_t qx = __float_as_uint(t.x), qy = __float_as_uint(t.y);
    // sign of sin: bit 1 of n; sign of cos: bit 1 of n + 1
    const uint32_t ssx = (qx << 30) & 0x80000000u, ssy = (qy << 30) & 0x80000000u;
    const uint32_t csx = ((qx + 1u) << 30) & 0x80000000u, csy = ((qy + 1u) << 30) & 0x80000000u;
    s.x = __uint_as_float(__float_as_uint((qx & 1u) ? cy.x : sy.x) ^ ssx);
    c.x = __uint_as_float(__float_as_uint((qx & 1u) ? sy.x : cy.x) ^ csx);
    s.y = __uint_as_float(__float_as_uint((qy & 1u) ? cy.y : sy.y) ^ ssy);
    c.y = __uint_as_float(__float_as_uint((qy & 1u) ? sy.y : cy.y) ^ csy);
}

// e^{i kappa r} / r without its 1/(4 pi), for CNT sources (as tc_eval16):
// the reciprocal square root as in the real path (0 for masked sources and,
// on touching leaves, for r^2 <= FLT_MIN), r = r^2 / r corrected by one
// Newton step, then tc_sincos2 of kappa r. A zero reciprocal gives
// kappa r = 0 (not the NaN of +inf * 0), so masked sources have the value 0.
template <bool ADJ, int CNT, int AX>
__device__ __forceinline__ void tc_ceval(const float* c, const float4* xl, int j0, float4 nt, float4 nl,
                                         float kappa, uint32_t* grh, uint32_t* grl, uint32_t* gih, uint32_t* gil) {
    const float2 ntx = tc_f2(nt.x), nty = tc_f2(nt.y), ntz = tc_f2(nt.z);
    float2 nlx, nly, nlz;
    if (ADJ) nlx = tc_f2(nl.x), nly = tc_f2(nl.y), nlz = tc_f2(nl.z);
    const float2 m1 = tc_f2(-1.f), split = tc_f2(8193.f), kap = tc_f2(kappa), half = tc_f2(0.5f);
#pragma unroll
    for (int q = 0; q < CNT / 4; ++q) {
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
            const float2 ri = make_float2(tc_green<1, ADJ>(r2.x), tc_green<1, ADJ>(r2.y));
            float2 r = __fmul2_rn(r2, ri);
            r = __ffma2_rn(__fmul2_rn(half, ri), __ffma2_rn(__fmul2_rn(r, m1), r, r2), r);
            float2 kr = __fmul2_rn(kap, r);
            kr.x = ri.x > 0.f ? kr.x : 0.f;
            kr.y = ri.y > 0.f ? kr.y : 0.f;
            float2 sn, cs;
            tc_sincos2(kr, sn, cs);
            const float2 gR = __fmul2_rn(cs, ri), gI = __fmul2_rn(sn, ri);
            // Veltkamp's split of both parts (as tc_eval16)
            const float2 tR = __fmul2_rn(gR, split), tI = __fmul2_rn(gI, split);
            const float2 hR = __ffma2_rn(__ffma2_rn(gR, m1, tR), m1, tR);
            const float2 hI = __ffma2_rn(__ffma2_rn(gI, m1, tI), m1, tI);
            const float2 lR = __ffma2_rn(hR, m1, gR), lI = __ffma2_rn(hI, m1, gI);
            grh[jj] = __float_as_uint(hR.x), grh[jj + 1] = __float_as_uint(hR.y);
            grl[jj] = __float_as_uint(lR.x), grl[jj + 1] = __float_as_uint(lR.y);
            gih[jj] = __float_as_uint(hI.x), gih[jj + 1] = __float_as_uint(hI.y);
            gil[jj] = __float_as_uint(lI.x), gil[jj + 1] = __float_as_uint(lI.y);
        }
    }
}

// One CTA per tensor-core item, the roles and barriers of tc_near_kernel
// (kComputeC compute threads); 16 complex right-hand sides per pass
// (a.r0 .. a.r0 + 15), U complex64 rows.
template <int NS = kNSC>
__global__ void __launch_bounds__(kThreadsC, 1) tc_cnear_kernel(const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSharedC<NS>& S = *reinterpret_cast<TcSharedC<NS>*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const TcItem* itp = a.items + blockIdx.x;
    const int64_t row_off = itp->row_off;
    const int nrows = itp->nrows, nslot = itp->nslot, list_lo = itp->list_lo;
    const int ntile = itp->list_hi - list_lo;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sm_addr(&S.full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(sm_addr(&S.afull[s])), "r"(kComputeC));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sm_addr(&S.empty[s])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(sm_addr(&S.tmem)), "r"(kTmemColsC));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = S.tmem;
    bool err = false;

    if (warp == kComputeC / 32) {
        // ---------------- producer warp ----------------
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
                    const uint32_t bar = sm_addr(&S.full[s]);
                    mbar_arrive_tx(bar, 4u * kChunkFloatsC + 64u);
                    bulk_g2s_hint(sm_addr(S.st[s].bhi), a.B + (int64_t)chunk * kChunkFloatsC, 4u * kChunkFloatsC, bar,
                                  l2_evict_last());
                    bulk_g2s_hint(sm_addr(&S.st[s].tile), a.tiles + list_lo + t, 64u, bar, l2_evict_first());
                    if (hold && !mbar_wait(bar, 0u, a.wait_ns)) err = true;
                }
                __syncwarp();
            }
        }
        if (lane == 0) {
            for (int t = (ntile > NS ? ntile - NS : 0); t < ntile; ++t)
                if (!mbar_wait(sm_addr(&S.full[t % NS]), (uint32_t)((t / NS) & 1), a.wait_ns)) err = true;
        }
    } else if (warp == kComputeC / 32 + 1) {
        // ---------------- MMA issuer (one thread) ----------------
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                                   ((128u >> 4) << 24);
            for (int m = 0; m < ntile; ++m) {
                const int s = m % NS, ab = m % kNA;
                if (!mbar_wait(sm_addr(&S.afull[s]), (uint32_t)((m / NS) & 1), a.wait_ns)) err = true;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t bh = sm_addr(S.st[s].bhi), bl = sm_addr(S.st[s].blo);
                const uint32_t bph = sm_addr(S.st[s].bphi), bpl = sm_addr(S.st[s].bplo);
                const uint32_t d = tbase + kColD + 32u * (m & 1);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t arh = tbase + kColAc + 128u * ab + 8u * k, arl = arh + 32u;
                    const uint32_t aih = arh + 64u, ail = arh + 96u;
                    const uint32_t ko = 2u * kBLbo * k;
                    mma_tf32(d, arh, smem_desc(bh + ko), idesc, k > 0 ? 1u : 0u);
                    mma_tf32(d, arh, smem_desc(bl + ko), idesc, 1u);
                    mma_tf32(d, arl, smem_desc(bh + ko), idesc, 1u);
                    mma_tf32(d, aih, smem_desc(bph + ko), idesc, 1u);
                    mma_tf32(d, aih, smem_desc(bpl + ko), idesc, 1u);
                    mma_tf32(d, ail, smem_desc(bph + ko), idesc, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(sm_addr(&S.empty[s])) : "memory");
            }
        }
    } else {
        // ---------------- compute warps: thread (row, quarter) ----------------
        const int row = tid & 127, quarter = tid >> 7;
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
        const int r_first = 32 * (warp & 3), r_last = min(r_first + 31, nrows - 1);
        int s_lo = 0, s_hi = 0;
        for (int c = 1; c < nslot; ++c) {
            if (r_first >= itp->slot_start[c]) s_lo = c;
            if (r_last >= itp->slot_start[c]) s_hi = c;
        }
        const int nsw = max(1, s_hi - s_lo + 1);
        const int myloc = min(max(myslot - s_lo, 0), kMaxSlots - 1);
        float* wc = S.wc[warp];
        constexpr uint32_t kKeepMask = (1u << kSrcC) - 1u;
        const int j0 = kSrcC * quarter;
        float acc[kColsC];
#pragma unroll
        for (int c = 0; c < kColsC; ++c) {
            acc[c] = 0.f;
            S.outer[c][tid] = 0.f;
        }
        auto drain = [&](int m) {
            if (!mbar_wait(sm_addr(&S.empty[m % NS]), (uint32_t)((m / NS) & 1), a.wait_ns)) err = true;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t v[kColsC];
            tmem_ld8(tbase + lane_off + kColD + 32u * (m & 1) + (uint32_t)(kColsC * quarter), v);
#pragma unroll
            for (int c = 0; c < kColsC; ++c) acc[c] += __uint_as_float(v[c]);
            if (m % kTcGroup == kTcGroup - 1) {
#pragma unroll
                for (int c = 0; c < kColsC; ++c) {
                    S.outer[c][tid] += acc[c];
                    acc[c] = 0.f;
                }
            }
        };
        for (int u = 0; u < ntile; ++u) {
            const int s = u % NS;
            if (!mbar_wait(sm_addr(&S.full[s]), (uint32_t)((u / NS) & 1), a.wait_ns)) err = true;
            TcStageC& st = S.st[s];
            const bool adj = (st.tile.flags & TASK_ADJ) != 0;
            const float cx = st.tile.cen[0], cy = st.tile.cen[1], cz = st.tile.cen[2];
            const float4 nt = adj ? make_float4(cx - tx.x, cy - tx.y, cz - tx.z, 0.f)
                                  : make_float4((cx - tx.x) - tl.x, (cy - tx.y) - tl.y, (cz - tx.z) - tl.z, 0.f);
            const uint32_t keep = valid ? (st.tile.keep[myslot] >> j0) & kKeepMask : 0u;
            __syncwarp();
            for (int p = lane; p < nsw * kSrcC; p += 32) {
                const int ls = p / kSrcC, jj = p % kSrcC;
                const float4 v = st.xh[j0 + jj];
                const bool kept = ((st.tile.keep[s_lo + ls] >> (j0 + jj)) & 1u) != 0u;
                float* d = wc + ls * kSlotFloatsC + jj;
                d[0] = kept ? v.x : kFar;
                d[kSrcC] = kept ? v.y : kFar;
                d[2 * kSrcC] = kept ? v.z : kFar;
            }
            __syncwarp();
            if (u >= 2) drain(u - 2);
            const uint32_t acol = tbase + lane_off + kColAc + 128u * (u % kNA) + (uint32_t)j0;
            const float* c = wc + myloc * kSlotFloatsC;
            const bool none = __all_sync(0xffffffffu, keep == 0);
            uint32_t grh[kSrcC], grl[kSrcC], gih[kSrcC], gil[kSrcC];
            if (none) {
#pragma unroll
                for (int jj = 0; jj < kSrcC; ++jj) grh[jj] = grl[jj] = gih[jj] = gil[jj] = 0u;
            } else if (adj) {
                tc_ceval<true, kSrcC, kSrcC>(c, st.xl, j0, nt, nl, a.kappa, grh, grl, gih, gil);
            } else {
                tc_ceval<false, kSrcC, kSrcC>(c, st.xl, j0, nt, nl, a.kappa, grh, grl, gih, gil);
            }
            tmem_st8(acol, grh);
            tmem_st8(acol + 32u, grl);
            tmem_st8(acol + 64u, gih);
            tmem_st8(acol + 96u, gil);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(sm_addr(&S.afull[s]));
        }
        for (int m = (ntile >= 2 ? ntile - 2 : 0); m < ntile; ++m) drain(m);
#pragma unroll
        for (int c = 0; c < kColsC; ++c) acc[c] += S.outer[c][tid];
        if (valid) {
            // quarter q holds columns 8q .. 8q + 7: real parts of right-hand
            // sides r0 + 8 (q & 1) .. + 7 (q < 2), their imaginary parts (q >= 2)
            const float scale = (float)green_scale<2>();
            const int64_t base = (row_off + row) * a.nrhs;
            const int c0 = a.r0 + kColsC * (quarter & 1), part = quarter >> 1;
#pragma unroll
            for (int c = 0; c < kColsC; ++c)
                if (c0 + c < a.nrhs) a.U[2 * (base + c0 + c) + part] = scale * acc[c];
        }
    }
    if (err) atomicExch(a.status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(kTmemColsC));
    }
}

}  // namespace skel
