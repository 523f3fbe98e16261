// Upward and downward passes of Algorithm 2 on the tensor cores (FP32_TC,
// real kernels): the skeleton GEMMs qhat_S = q_S + T q_R and u_R += T^* uhat
// of a level as split-TF32 MMAs (tcgen05, kind::tf32) over 32 right-hand
// sides at a time. Opt-in (skel_options.updown_tc): see the accuracy note
// below.
//
// Work item: one box of the level and up to 128 of its output rows (upward:
// skeleton rows i < k; downward: redundant rows j < |I_B| - k). The inner
// index (upward j < |I_B| - k, downward i < k) runs in tiles of 32. T is
// static, so the plan keeps each item's A operand in tile order, one blob
// per tile: its nrows x 32 values in the quad layout of the per-tile store
// (value (row, 4 q + e) of column half h at float ((4 h + q) nrows + row) * 4
// + e; zero past the inner size), then the 32 entry indices whose rows of X
// form the tile's B operand (-1 past the inner size). The producer warp
// bulk-copies a tile's blob into a stage; the compute warps read their row's
// 16 values, split them into three TF32 parts and write A to tensor memory,
// and build the B operand (the tile's 32 rows of X for this pass's 32
// columns, three parts, in the shared-memory layout of the MMA) from the
// entries; the MMA warp forms each tile's product in one of two tensor-memory
// accumulators and the compute warps add the tiles in FP32 registers.
// Split: x = hi + mid + lo with hi = tf32(x), mid = tf32(x - hi) (both
// rounded to nearest) and lo = x - hi - mid (at most 2 significant bits,
// exact in TF32); the 6 products hh, hm, mh, hl, lh, mm (24 MMAs per tile)
// leave out terms below 2^-33 of the product. Accuracy: the skeleton sums
// cancel (T mixes signs), and the tensor core's accumulation is less accurate
// than FP32 FMAs on them: relative error 1.3e-6 instead of 7.8e-7 at
// N = 2^20, tol 1e-6, with this split as with the translations' two-part
// one, so the error comes from the accumulation. The epilogue writes
// qhat_S = q_S + D into the parent's slot (upward) or adds D to u_R
// (downward); the downward items of row 0 also add uhat to u_S.
//
// Every wait is bounded (the globaltimer limit of the translations): on
// timeout the kernel raises the status word and finishes the protocol; entry
// indices read from a stage are range-checked before use, so a stage that
// never landed can only give wrong values, not a wrong address.
#pragma once

#include "tc_kernels.cuh"

namespace skel {

struct UdItem {                                // 24 bytes
    int64_t a_off;                             // float offset of its first tile blob
    int32_t box;                               // index into the level's UpBox array (dp->up)
    int32_t row0;                              // first output row
    int32_t nrows;                             // output rows (0..128)
    int32_t ntile;                             // inner tiles of 32
};
static_assert(sizeof(UdItem) == 24, "UdItem layout");

struct UdArgs {
    const UdItem* items;
    const UpBox* up;
    const int32_t* pos;
    const float* A;                            // the tile blobs
    float* X;                                  // Q (upward) or U (downward), rows of nrhs
    int64_t n_tot;                             // entries (range check of the blob indices)
    int nrhs;
    int r0;                                    // first right-hand side of this pass
    int* status;
    uint64_t wait_ns;
};

// blob of a tile with nrows output rows: nrows x 32 floats, then 32 int32
__host__ __device__ constexpr int64_t ud_blob_floats(int nrows) { return (int64_t)nrows * 32 + 32; }

// x = hi + mid + lo, each a TF32 value (see above)
__device__ __forceinline__ void tf32_split3(float x, float& hi, float& mid, float& lo) {
    hi = __uint_as_float(to_tf32(x));
    const float r = x - hi;
    mid = __uint_as_float(to_tf32(r));
    lo = r - mid;
}

constexpr int kUdNST = 3;                      // stages
struct alignas(128) UdStage {
    float4 ga[kTileFloats / 4 + 8];            // the tile blob (values, then entry indices)
    float b[3 * 1024];                         // B hi, mid, lo (written by the compute warps)
};
static_assert(sizeof(float4) * (kTileFloats / 4 + 8) % 128 == 0, "B area 128-byte aligned");
struct UdShared {
    UdStage st[kUdNST];
    uint64_t full[kUdNST], afull[kUdNST], empty[kUdNST];
    uint32_t tmem;
};
constexpr int kUdSmemRequest = 100 * 1024;    // two CTAs per SM
static_assert(sizeof(UdShared) <= kUdSmemRequest, "shared memory plan (up/down)");
// tensor memory: accumulators D0, D1 at [0, 64), A[b] hi, mid, lo at 64 + 96 b + 0 / 32 / 64 (b < 2)
constexpr uint32_t kUdColA = 64;

template <bool DOWN>
__global__ void __launch_bounds__(kTcThreads, 2) tc_ud_kernel(const UdArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    UdShared& S = *reinterpret_cast<UdShared*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const UdItem it = a.items[blockIdx.x];
    const UpBox u = a.up[it.box];
    const int k = u.k;
    const int nrows = it.nrows, ntile = it.ntile;
    const int64_t blob = ud_blob_floats(nrows);

    if (tid == 0) {
        for (int s = 0; s < kUdNST; ++s) {
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
        // ---------------- producer warp: the tile blobs, kUdNST ahead ----------------
        if (lane == 0) {
            const float* src = a.A + it.a_off;
            const uint32_t bytes = (uint32_t)(blob * 4);
            for (int t = 0; t < ntile; ++t) {
                const int s = t % kUdNST;
                if (t >= kUdNST && !mbar_wait(sm_addr(&S.empty[s]), (uint32_t)(((t - kUdNST) / kUdNST) & 1), a.wait_ns))
                    err = true;
                const uint32_t bar = sm_addr(&S.full[s]);
                mbar_arrive_tx(bar, bytes);
                bulk_g2s_hint(sm_addr(S.st[s].ga), src + (int64_t)t * blob, bytes, bar, l2_evict_first());
            }
            // every copy has landed before the CTA may exit
            for (int t = (ntile > kUdNST ? ntile - kUdNST : 0); t < ntile; ++t)
                if (!mbar_wait(sm_addr(&S.full[t % kUdNST]), (uint32_t)((t / kUdNST) & 1), a.wait_ns)) err = true;
        }
    } else if (warp == kTcCompute / 32 + 1) {
        // ---------------- MMA issuer: tile m into accumulator m & 1 ----------------
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                                   ((128u >> 4) << 24);
            for (int m = 0; m < ntile; ++m) {
                const int s = m % kUdNST;
                if (!mbar_wait(sm_addr(&S.afull[s]), (uint32_t)((m / kUdNST) & 1), a.wait_ns)) err = true;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t bh = sm_addr(S.st[s].b), bm = bh + 4u * 1024u, bl = bh + 8u * 1024u;
                const uint32_t d = tbase + kColD + 32u * (m & 1);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t ah = tbase + kUdColA + 96u * (m & 1) + 8u * kk, am = ah + 32u, al = ah + 64u;
                    const uint32_t ko = 2u * kBLbo * kk;
                    mma_tf32(d, ah, smem_desc(bh + ko), idesc, kk > 0 ? 1u : 0u);
                    mma_tf32(d, ah, smem_desc(bm + ko), idesc, 1u);
                    mma_tf32(d, am, smem_desc(bh + ko), idesc, 1u);
                    mma_tf32(d, ah, smem_desc(bl + ko), idesc, 1u);
                    mma_tf32(d, al, smem_desc(bh + ko), idesc, 1u);
                    mma_tf32(d, am, smem_desc(bm + ko), idesc, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(sm_addr(&S.empty[s])) : "memory");
            }
        }
    } else {
        // ---------------- compute warps ----------------
        const int row = tid & 127, half = tid >> 7;          // A: thread (row, column half)
        const int n = tid & 31, jq = tid >> 5;               // B: column n, inner rows 4 jq .. 4 jq + 3
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        const bool valid = row < nrows;
        const int bcol = a.r0 + n;
        // this thread's four B values of tile t (its stage has landed)
        auto load_b = [&](int t, float* x) {
            const int* ids = reinterpret_cast<const int*>(S.st[t % kUdNST].ga) + nrows * 32;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int e = ids[4 * jq + c];
                x[c] = (e >= 0 && e < a.n_tot && bcol < a.nrhs) ? a.X[(int64_t)e * a.nrhs + bcol] : 0.f;
            }
        };
        const int c0 = a.r0 + 16 * half;
        if (DOWN && it.row0 == 0) {
            // u_S += uhat (this pass's columns), once per box: thread (row,
            // half) takes rows row, row + 128, ... and its 16 columns, every
            // load of a row issued before its stores
            for (int i = row; i < k; i += 128) {
                const int64_t es = (u.off + a.pos[u.off + i]) * a.nrhs, eh = (u.dst + i) * a.nrhs;
                float us[16], uh[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const bool ok = c0 + c < a.nrhs;
                    us[c] = ok ? a.X[es + c0 + c] : 0.f;
                    uh[c] = ok ? a.X[eh + c0 + c] : 0.f;
                }
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    if (c0 + c < a.nrhs) a.X[es + c0 + c] = us[c] + uh[c];
            }
        }
        float acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = 0.f;
        auto drain = [&](int m) {                            // add tile m's product (its MMAs are done)
            if (!mbar_wait(sm_addr(&S.empty[m % kUdNST]), (uint32_t)((m / kUdNST) & 1), a.wait_ns)) err = true;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t v[16];
            tmem_ld16(tbase + lane_off + kColD + 32u * (m & 1) + 16u * half, v);
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] += __uint_as_float(v[c]);
        };
        float xc[4] = {0.f, 0.f, 0.f, 0.f}, xn[4] = {0.f, 0.f, 0.f, 0.f};
        if (ntile > 0) {
            if (!mbar_wait(sm_addr(&S.full[0]), 0u, a.wait_ns)) err = true;
            load_b(0, xc);
        }
        for (int t = 0; t < ntile; ++t) {
            const int s = t % kUdNST;
            // the next tile's B rows go out now and arrive while this one is processed
            if (t + 1 < ntile) {
                if (!mbar_wait(sm_addr(&S.full[(t + 1) % kUdNST]), (uint32_t)(((t + 1) / kUdNST) & 1), a.wait_ns))
                    err = true;
                load_b(t + 1, xn);
            }
            // B of tile t in three parts, in the layout of tc_bprep_kernel
            {
                float4 h, m, l;
                tf32_split3(xc[0], h.x, m.x, l.x);
                tf32_split3(xc[1], h.y, m.y, l.y);
                tf32_split3(xc[2], h.z, m.z, l.z);
                tf32_split3(xc[3], h.w, m.w, l.w);
                float* bb = S.st[s].b + jq * 128 + n * 4;
                *reinterpret_cast<float4*>(bb) = h;
                *reinterpret_cast<float4*>(bb + 1024) = m;
                *reinterpret_cast<float4*>(bb + 2048) = l;
            }
            // A of tile t: this row's 16 values of column half `half`
            uint32_t gh[16], gm[16], gl[16];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int quad = 4 * half + q;
                const float4 g4 = valid ? S.st[s].ga[quad * nrows + row] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float h, m, l;
                    tf32_split3(gv[e], h, m, l);
                    gh[4 * q + e] = __float_as_uint(h);
                    gm[4 * q + e] = __float_as_uint(m);
                    gl[4 * q + e] = __float_as_uint(l);
                }
            }
            // A buffer and accumulator t & 1 were last used by tile t - 2
            if (t >= 2) drain(t - 2);
            const uint32_t acol = tbase + lane_off + kUdColA + 96u * (t & 1) + 16u * half;
            tmem_st16(acol, gh);
            tmem_st16(acol + 32u, gm);
            tmem_st16(acol + 64u, gl);
            // the B stores are generic-proxy writes that the tensor core reads
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(sm_addr(&S.afull[s]));
#pragma unroll
            for (int c = 0; c < 4; ++c) xc[c] = xn[c];
        }
        for (int m = (ntile >= 2 ? ntile - 2 : 0); m < ntile; ++m) drain(m);
        if (valid) {
            const int i = it.row0 + row;
            if (!DOWN) {
                // qhat_S = q_S + T q_R into the parent's slot
                const int64_t es = (u.off + a.pos[u.off + i]) * a.nrhs, ed = (u.dst + i) * a.nrhs;
                float qs[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) qs[c] = c0 + c < a.nrhs ? a.X[es + c0 + c] : 0.f;
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    if (c0 + c < a.nrhs) a.X[ed + c0 + c] = qs[c] + acc[c];
            } else {
                // u_R += T^* uhat
                const int64_t ed = (u.off + a.pos[u.off + k + i]) * a.nrhs;
                float ur[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) ur[c] = c0 + c < a.nrhs ? a.X[ed + c0 + c] : 0.f;
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    if (c0 + c < a.nrhs) a.X[ed + c0 + c] = ur[c] + acc[c];
            }
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
