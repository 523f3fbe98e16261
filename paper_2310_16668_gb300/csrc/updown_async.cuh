// Upward / downward passes (FP32), the CTA-wide form: a CTA owns 32 NW
// output rows (NW warps, 32 rows each; a thread holds 4 rows x 8 right-hand
// sides) x 32 right-hand sides of one box and streams the inner index in chunks of 32
// through a two-stage pipeline of asynchronous copies that all its threads
// issue: per chunk the A block (32 inner x 32 NW rows, zero-filled past the
// box) and the chunk's 32 rows of X (shared by the warps). The chunks are
// taken in stream order (stream s: chunks s, s + NS, ...), each stream summed
// on its own and the streams added in order, which is exactly the arithmetic
// of updown_kernel with one warp per CTA: every launch shape of both kernels
// gives the same bits, so the autotuner may pick any of them per level. The
// entry indices of the chunk after next are loaded while the current chunk's
// copies are waited for. VEC: 16-byte copies, from a copy of T whose columns
// are padded to a multiple of 4 floats (zeros) and start 16-byte aligned
// (toff: per box, its first float), and B rows of 32 columns (nrhs a
// multiple of 4); else 4-byte copies from T itself.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "skel_kernels.cuh"

namespace skel {

__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" :: "r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory");
}

constexpr int kUdrStages = 2;
// dynamic shared memory: per stage the A block (32 x 32 NW) and the B block (32 x 32)
__host__ __device__ constexpr int ud_rows_smem(int NW) {
    return kUdrStages * (NW + 1) * kGT * kGT * (int)sizeof(float);
}

// The CTAs come from a work list of (box, first output row) pairs, one per
// 32 NW rows of each box of the level (a downward box without redundant rows
// keeps one, for its u_S += uhat): in adaptive trees the boxes of a level
// differ widely in size, and a grid sized by the largest would launch
// mostly empty CTAs.
template <bool DOWN, int NW, bool VEC>
__global__ void __launch_bounds__(32 * NW) updown_rows_kernel(const UpBox* __restrict__ up,
                                                              const int2* __restrict__ work,
                                                              const int32_t* __restrict__ pos,
                                                              const float* __restrict__ T,
                                                              const int64_t* __restrict__ toff, float* X, int nrhs) {
    constexpr int NS = ud_streams<float>();
    constexpr int ROWS = 32 * NW;
    constexpr int STAGE = (NW + 1) * kGT * kGT;           // floats per stage: A then B
    static_assert(NW == 1 || NW == 2 || NW == 4 || NW == 8, "warps per CTA");
    extern __shared__ __align__(16) unsigned char udr_raw[];
    float* sm = reinterpret_cast<float*>(udr_raw);
    const int2 wi = work[blockIdx.x];
    const UpBox u = up[wi.x];
    const int k = u.k, r = u.n - u.k;
    const int nout = DOWN ? r : k, ninner = DOWN ? k : r;
    const int row0 = wi.y, c0 = blockIdx.z * kGT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int col = c0 + lane;
    const bool colok = col < nrhs;
    if (DOWN && row0 == 0 && colok) {                    // u_S += uhat, this CTA's columns
        for (int i0 = warp; i0 < k; i0 += 8 * NW) {
            float uh[8], us[8];
            int64_t at[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = i0 + q * NW;
                at[q] = -1;
                if (i < k) {
                    at[q] = (u.off + pos[u.off + i]) * nrhs + col;
                    uh[q] = X[(u.dst + i) * nrhs + col];
                    us[q] = X[at[q]];
                }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (at[q] >= 0) X[at[q]] = us[q] + uh[q];
        }
    }
    if (row0 >= nout) return;
    const int nch = (ninner + kGT - 1) / kGT;
    const int nsum = nch < NS ? nch : NS;
    const bool arow = row0 + tid < nout;                  // this thread's A row (copies)
    // the entry of B row `lane` of chunk ch (lanes past the chunk: 0, unused)
    auto entry = [&](int ch) -> int64_t {
        const int j0 = ch * kGT, jn = min(kGT, ninner - j0);
        if (lane >= jn) return 0;
        return DOWN ? (u.dst + j0 + lane) : (u.off + pos[u.off + k + j0 + lane]);
    };
    const int ld = VEC ? (nout + 3) & ~3 : nout;         // column stride of this box's block
    const int64_t t0 = VEC ? toff[wi.x] : u.T_off;
    // the copies of chunk ch into stage buf: A (inner jj, row tid), B rows jj = warp, warp + NW, ...
    auto issue = [&](int ch, int64_t ri, float* buf) {
        const int j0 = ch * kGT, jn = min(kGT, ninner - j0);
        const uint32_t sa = (uint32_t)__cvta_generic_to_shared(buf);
        if constexpr (VEC) {
            // A: 32 columns x ROWS / 4 segments of 4 rows; B: 32 rows x 8 segments
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int idx = tid + m * ROWS, jj = idx / (ROWS / 4), r4 = (idx % (ROWS / 4)) * 4;
                const bool av = jj < jn && row0 + r4 < ld;
                const float* ga = av ? T + t0 + row0 + r4 + (int64_t)(j0 + jj) * ld : T;
                cp_async16(sa + (uint32_t)(jj * ROWS + r4) * 4u, ga, av ? 16u : 0u);
            }
            for (int idx = tid; idx < kGT * 8; idx += ROWS) {
                const int jj = idx >> 3, c = c0 + (idx & 7) * 4;
                const int64_t rj = __shfl_sync(0xffffffffu, ri, jj);
                const int nb = jj < jn ? max(0, min(16, (nrhs - c) * 4)) : 0;
                const float* gb = nb > 0 ? X + rj * nrhs + c : X;
                cp_async16(sa + (uint32_t)(kGT * ROWS + jj * kGT + (idx & 7) * 4) * 4u, gb, (uint32_t)nb);
            }
        } else {
#pragma unroll 8
            for (int jj = 0; jj < kGT; ++jj) {
                const bool av = jj < jn && arow;
                const float* ga = av ? T + t0 + row0 + tid + (int64_t)(j0 + jj) * ld : T;
                cp_async4(sa + (uint32_t)(jj * ROWS + tid) * 4u, ga, av ? 4u : 0u);
            }
#pragma unroll
            for (int m = 0; m < kGT / NW; ++m) {
                const int jj = warp + m * NW;
                const int64_t rj = __shfl_sync(0xffffffffu, ri, jj);
                const bool bv = jj < jn && colok;
                const float* gb = bv ? X + rj * nrhs + col : X;
                cp_async4(sa + (uint32_t)(kGT * ROWS + jj * kGT + lane) * 4u, gb, bv ? 4u : 0u);
            }
        }
    };
    // chunks in stream order: (stream, chunk) -> the next one
    auto advance = [&](int& s, int& ch) {
        if (ch + NS < nch) ch += NS;
        else ch = ++s;
    };
    const int rg = lane & 7, cg = lane >> 3;             // compute: 4 rows x 8 columns per thread
    float acc[kGT], tot[kGT];                            // element (r, c) at 8 r + c
#pragma unroll
    for (int i = 0; i < kGT; ++i) acc[i] = tot[i] = 0.f;
    if (nch > 0) {
        // issue pointer (stream, chunk) and the entries of its chunk
        int is = 0, ic = 0;
        int64_t ri = entry(0);
        for (int p = 0; p < kUdrStages - 1; ++p) {
            if (is < nsum) {
                issue(ic, ri, sm + p * STAGE);
                advance(is, ic);
                ri = is < nsum ? entry(ic) : 0;
            }
            cp_async_commit();
        }
        int cs = 0, cc = 0;                              // compute pointer
        for (int t = 0; t < nch; ++t) {
            if (is < nsum) {
                issue(ic, ri, sm + ((t + kUdrStages - 1) % kUdrStages) * STAGE);
                advance(is, ic);
                ri = is < nsum ? entry(ic) : 0;
            }
            cp_async_commit();
            cp_async_wait<kUdrStages - 1>();
            __syncthreads();
            const float* As = sm + (t % kUdrStages) * STAGE + warp * kGT + 4 * rg;
            const float* Bs = sm + (t % kUdrStages) * STAGE + kGT * ROWS + 8 * cg;
            // thread (rg, cg): rows 4 rg .. + 3 of the warp's 32, columns
            // 8 cg .. + 7; each element gets the same FMA chain as in
            // updown_kernel (one FMA per inner index, in order)
#pragma unroll 4
            for (int jj = 0; jj < kGT; ++jj) {
                const float4 a = *reinterpret_cast<const float4*>(As + jj * ROWS);
                const float4 b0 = *reinterpret_cast<const float4*>(Bs + jj * kGT);
                const float4 b1 = *reinterpret_cast<const float4*>(Bs + jj * kGT + 4);
                const float av[4] = {a.x, a.y, a.z, a.w};
                const float2 bp[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                                      make_float2(b1.z, b1.w)};
                float2* acc2 = reinterpret_cast<float2*>(acc);
#pragma unroll
                for (int r4 = 0; r4 < 4; ++r4) {
                    const float2 a2 = make_float2(av[r4], av[r4]);
#pragma unroll
                    for (int c2 = 0; c2 < 4; ++c2) acc2[r4 * 4 + c2] = __ffma2_rn(a2, bp[c2], acc2[r4 * 4 + c2]);
                }
            }
            if (!(cc + NS < nch)) {                      // the stream's last chunk
#pragma unroll
                for (int i = 0; i < kGT; ++i) {
                    tot[i] = cs == 0 ? acc[i] : tot[i] + acc[i];
                    acc[i] = 0.f;
                }
            }
            advance(cs, cc);
            __syncthreads();                             // before this stage is filled again
        }
    }
    // this thread's 4 rows x 8 columns: every old value is loaded before the stores
    const int cb = c0 + 8 * cg;
    int64_t src[4], dst[4];
#pragma unroll
    for (int r4 = 0; r4 < 4; ++r4) {
        const int orow = row0 + warp * kGT + 4 * rg + r4;
        dst[r4] = -1;
        if (orow < nout && cb < nrhs) {
            src[r4] = DOWN ? (u.off + pos[u.off + k + orow]) * nrhs : (u.off + pos[u.off + orow]) * nrhs;
            dst[r4] = DOWN ? src[r4] : (u.dst + orow) * nrhs;
        }
    }
    float old[kGT];
#pragma unroll
    for (int r4 = 0; r4 < 4; ++r4)
#pragma unroll
        for (int c = 0; c < 8; ++c)
            old[8 * r4 + c] = (dst[r4] >= 0 && cb + c < nrhs) ? X[src[r4] + cb + c] : 0.f;
#pragma unroll
    for (int r4 = 0; r4 < 4; ++r4)
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (dst[r4] >= 0 && cb + c < nrhs) X[dst[r4] + cb + c] = old[8 * r4 + c] + tot[8 * r4 + c];
}

}  // namespace skel
