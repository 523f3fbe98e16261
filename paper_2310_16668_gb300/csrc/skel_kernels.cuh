// CUDA-core kernels of the apply (FP64 and FP32): permutation, upward and
// downward interpolation (Algorithm 2, outgoing / incoming representations)
// and the near-field translation kernel.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "host.h"

namespace skel {

// ---- scalar types ------------------------------------------------------------
template <class R>
struct alignas(2 * sizeof(R)) Cx {
    R x, y;
};
template <class R> __host__ __device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <class R> __host__ __device__ __forceinline__ Cx<R>& operator+=(Cx<R>& a, Cx<R> b) { a.x += b.x; a.y += b.y; return a; }
template <class R> __host__ __device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class R> __host__ __device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) { return {s * a.x, s * a.y}; }
template <class R> __host__ __device__ __forceinline__ Cx<R> conj(Cx<R> a) { return {a.x, -a.y}; }
__host__ __device__ __forceinline__ float conj(float a) { return a; }
__host__ __device__ __forceinline__ double conj(double a) { return a; }
template <class S> __device__ __forceinline__ S zero();
template <> __device__ __forceinline__ float zero<float>() { return 0.f; }
template <> __device__ __forceinline__ double zero<double>() { return 0.0; }
template <> __device__ __forceinline__ Cx<float> zero<Cx<float>>() { return {0.f, 0.f}; }
template <> __device__ __forceinline__ Cx<double> zero<Cx<double>>() { return {0.0, 0.0}; }

template <class R> struct RealT;
template <> struct RealT<float> { using V4 = float4; };
template <> struct RealT<double> { using V4 = double4; };
template <class R, bool C> struct Scal { using T = R; };
template <class R> struct Scal<R, true> { using T = Cx<R>; };

__device__ __forceinline__ float shfl_down(float v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
template <class R> __device__ __forceinline__ Cx<R> shfl_down(Cx<R> v, int o) {
    return {shfl_down(v.x, o), shfl_down(v.y, o)};
}
template <class S> __device__ __forceinline__ S warp_sum(S v) {
    for (int o = 16; o > 0; o >>= 1) v += shfl_down(v, o);
    return v;
}

// ---- permutation ------------------------------------------------------------------
// q (user point order; each right-hand side a column of N) -> Q (entry space,
// one row of nrhs per entry). eop[p] = the leaf entry of user point p. A tile
// of 32 points x 32 right-hand sides goes through shared memory, so the
// column reads and the row writes are both contiguous.
// eop2 (may be null): for a point of a leaf box that keeps all its points as
// skeletons (k = |I_B|, no redundant index), the entry of its skeleton row in
// the parent's slot, else -1. Such a box's upward step is the copy
// qhat_S = q_S into that slot and its downward step the sum u_S + uhat_S;
// permute_in writes the second copy and permute_out adds the slot's value,
// so the level launches skip the box.
constexpr int kPermTile = 32;
constexpr int kPermThreads = 256;

template <class S>
__global__ void __launch_bounds__(kPermThreads) permute_in(const int64_t* __restrict__ eop,
                                                           const int64_t* __restrict__ eop2, const S* __restrict__ q,
                                                           S* __restrict__ Q, int64_t N, int nrhs) {
    __shared__ S t[kPermTile][kPermTile + 1];
    const int64_t p0 = (int64_t)blockIdx.x * kPermTile;
    const int r0 = blockIdx.y * kPermTile;
    const int tx = threadIdx.x % kPermTile, ty = threadIdx.x / kPermTile;
    for (int k = ty; k < kPermTile; k += kPermThreads / kPermTile)
        if (r0 + k < nrhs && p0 + tx < N) t[k][tx] = q[(int64_t)(r0 + k) * N + p0 + tx];
    __syncthreads();
    for (int k = ty; k < kPermTile; k += kPermThreads / kPermTile)
        if (p0 + k < N && r0 + tx < nrhs) {
            const S v = t[tx][k];
            Q[eop[p0 + k] * nrhs + r0 + tx] = v;
            if (eop2) {
                const int64_t e2 = eop2[p0 + k];
                if (e2 >= 0) Q[e2 * nrhs + r0 + tx] = v;
            }
        }
}

template <class S>
__global__ void __launch_bounds__(kPermThreads) permute_out(const int64_t* __restrict__ eop,
                                                            const int64_t* __restrict__ eop2, const S* __restrict__ U,
                                                            S* __restrict__ u, int64_t N, int nrhs) {
    __shared__ S t[kPermTile][kPermTile + 1];
    const int64_t p0 = (int64_t)blockIdx.x * kPermTile;
    const int r0 = blockIdx.y * kPermTile;
    const int tx = threadIdx.x % kPermTile, ty = threadIdx.x / kPermTile;
    for (int k = ty; k < kPermTile; k += kPermThreads / kPermTile)
        if (p0 + k < N && r0 + tx < nrhs) {
            S v = U[eop[p0 + k] * nrhs + r0 + tx];
            if (eop2) {
                const int64_t e2 = eop2[p0 + k];
                if (e2 >= 0) v = v + U[e2 * nrhs + r0 + tx];
            }
            t[k][tx] = v;
        }
    __syncthreads();
    for (int k = ty; k < kPermTile; k += kPermThreads / kPermTile)
        if (r0 + k < nrhs && p0 + tx < N) u[(int64_t)(r0 + k) * N + p0 + tx] = t[tx][k];
}

// few right-hand sides: one element per thread, points fastest (contiguous
// column reads / writes on the user side)
template <class S>
__global__ void permute_in_narrow(const int64_t* __restrict__ eop, const int64_t* __restrict__ eop2,
                                  const S* __restrict__ q, S* __restrict__ Q, int64_t N, int nrhs) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N * nrhs) return;
    const int64_t p = g % N, r = g / N;
    const S v = q[g];
    Q[eop[p] * nrhs + r] = v;
    if (eop2) {
        const int64_t e2 = eop2[p];
        if (e2 >= 0) Q[e2 * nrhs + r] = v;
    }
}

template <class S>
__global__ void permute_out_narrow(const int64_t* __restrict__ eop, const int64_t* __restrict__ eop2,
                                   const S* __restrict__ U, S* __restrict__ u, int64_t N, int nrhs) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N * nrhs) return;
    const int64_t p = g % N, r = g / N;
    S v = U[eop[p] * nrhs + r];
    if (eop2) {
        const int64_t e2 = eop2[p];
        if (e2 >= 0) v = v + U[e2 * nrhs + r];
    }
    u[g] = v;
}

// ---- upward / downward passes ------------------------------------------------------------
// Upward (qhat_S = q_S + T q_R into the parent's slot): output rows i < k,
// inner index j < r, A(i, j) = T[i + j k] (T column-major k x r), B row j =
// the q row of R entry j. Downward (u_S += uhat, then u_R += T^* uhat): output
// rows j < r, inner index i < k, A(j, i) = Tt[j + i r] (the transposed copy,
// column-major r x k), B row i = uhat_i (the parent's slot). conj_op applies
// the complex conjugate to A (T^* downward, conj(T) for the transposed apply).
//
// A CTA owns 32 output rows x 32 right-hand sides of one box (grid x: box,
// y: row block, z: column block) and has W warps. The inner index runs in
// chunks of 32 dealt round-robin to NS streams (stream s: chunks s, s + NS,
// ...); warp w forms the partial sums of streams w, w + W, ... one after the
// other, each over its chunks in order, and the stream partials are added in
// stream order (through shared memory when W > 1, in registers when W = 1).
// The result is therefore the same for every W, which the autotuner picks
// per level. Within a warp, lane = right-hand side: per chunk the warp stages
// its 32 x 32 block of A (inner-major; each load is one coalesced column of
// 32 rows) and its 32 B rows (each load one coalesced row) in shared memory;
// each inner index then costs 32 row FMAs per lane (paired in FP32), with the
// A column read as broadcast 16-byte words.
constexpr int kGT = 32;
template <class S> __host__ __device__ constexpr int ud_streams() {
    return sizeof(S) <= 4 ? 8 : sizeof(S) <= 8 ? 4 : 2;
}
// dynamic shared memory of a CTA with W warps: per warp its A and B blocks,
// then (W > 1) the stream partials
template <class S> __host__ __device__ constexpr int ud_smem(int W) {
    return (W * 2 + (W > 1 ? ud_streams<S>() : 0)) * kGT * kGT * (int)sizeof(S);
}
constexpr int kUdSmemMax = 96 * 1024;

template <class S> __device__ __forceinline__ void ud_rows(S* acc, const S* a, S q) {
#pragma unroll
    for (int r = 0; r < kGT; ++r) acc[r] += a[r] * q;
}
template <> __device__ __forceinline__ void ud_rows<float>(float* acc, const float* a, float q) {
    const float2 q2 = make_float2(q, q);
    float2* acc2 = reinterpret_cast<float2*>(acc);
#pragma unroll
    for (int r4 = 0; r4 < kGT / 4; ++r4) {
        const float4 v = reinterpret_cast<const float4*>(a)[r4];
        acc2[2 * r4] = __ffma2_rn(make_float2(v.x, v.y), q2, acc2[2 * r4]);
        acc2[2 * r4 + 1] = __ffma2_rn(make_float2(v.z, v.w), q2, acc2[2 * r4 + 1]);
    }
}

template <class S, bool DOWN, int W>
__global__ void __launch_bounds__(32 * W) updown_kernel(const UpBox* __restrict__ up, const int32_t* __restrict__ pos,
                                                        const S* __restrict__ T, S* X, int nrhs, bool conj_op) {
    constexpr int NS = ud_streams<S>();
    static_assert(W == 1 || W == 2 || W == 4 || W == 8, "warps per CTA");
    static_assert(W <= NS, "at most one warp per stream");
    extern __shared__ __align__(16) unsigned char ud_raw[];
    S* sm = reinterpret_cast<S*>(ud_raw);
    const UpBox u = up[blockIdx.x];
    const int k = u.k, r = u.n - u.k;
    const int nout = DOWN ? r : k, ninner = DOWN ? k : r;
    const int row0 = blockIdx.y * kGT, c0 = blockIdx.z * kGT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col = c0 + lane;
    const bool colok = col < nrhs;
    if (DOWN && blockIdx.y == 0 && colok) {              // u_S += uhat, this CTA's columns
        // batches of 8 rows: every load of a batch is issued before its stores
        // (X is read and written through the same pointer, so the compiler
        // would otherwise keep each load behind the previous row's store)
        for (int i0 = warp; i0 < k; i0 += 8 * W) {
            S uh[8], us[8];
            int64_t at[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = i0 + q * W;
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
    S* As = sm + warp * 2 * kGT * kGT;                     // this warp's A block [inner][row]
    S* Bs = As + kGT * kGT;                                // and B block [inner][column]
    S* Ps = sm + W * 2 * kGT * kGT;                        // stream partials [stream][row][column]
    const int nch = (ninner + kGT - 1) / kGT;
    const int nsum = nch < NS ? nch : NS;                  // streams that receive chunks
    const bool rowok = row0 + lane < nout;
    S acc[kGT];
    S tot[W == 1 ? kGT : 1];
    for (int st = warp; st < nsum; st += W) {
#pragma unroll
        for (int i = 0; i < kGT; ++i) acc[i] = zero<S>();
        for (int ch = st; ch < nch; ch += NS) {
            const int j0 = ch * kGT, jn = min(kGT, ninner - j0);
            // the B rows of this chunk: their entry indices, one per lane
            int64_t ri = 0;
            if (lane < jn) ri = DOWN ? (u.dst + j0 + lane) : (u.off + pos[u.off + k + j0 + lane]);
            // stage the A and B blocks: a group's loads all go out before its
            // stores to shared memory (one memory latency per group)
            constexpr int G = sizeof(S) <= 4 ? 32 : sizeof(S) <= 8 ? 16 : 8;
#pragma unroll
            for (int g0 = 0; g0 < kGT; g0 += G) {
                S ra[G], rb[G];
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    const int jj = g0 + q;
                    const int64_t rj = __shfl_sync(0xffffffffu, ri, jj);
                    ra[q] = zero<S>();
                    rb[q] = zero<S>();
                    if (jj < jn) {
                        if (rowok) ra[q] = T[u.T_off + row0 + lane + (int64_t)(j0 + jj) * nout];
                        if (colok) rb[q] = X[rj * nrhs + col];
                    }
                }
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    As[(g0 + q) * kGT + lane] = conj_op ? conj(ra[q]) : ra[q];
                    Bs[(g0 + q) * kGT + lane] = rb[q];
                }
            }
            __syncwarp();
#pragma unroll 4
            for (int jj = 0; jj < kGT; ++jj) ud_rows<S>(acc, As + jj * kGT, Bs[jj * kGT + lane]);
            __syncwarp();                                  // before the next chunk overwrites the blocks
        }
        if constexpr (W == 1) {
#pragma unroll
            for (int i = 0; i < kGT; ++i) tot[i] = st == 0 ? acc[i] : tot[i] + acc[i];
        } else {
#pragma unroll
            for (int i = 0; i < kGT; ++i) Ps[(st * kGT + i) * kGT + lane] = acc[i];
        }
    }
    if constexpr (W > 1) __syncthreads();
    if (!colok) return;
    // rows of this CTA: warp w writes rows w, w + W, ...
    if constexpr (W == 1) {
        if (nsum == 0) {
#pragma unroll
            for (int i = 0; i < kGT; ++i) tot[i] = zero<S>();
        }
    }
    // the rows this warp writes (w, w + W, ...): all their old values are
    // loaded before any store
    constexpr int R = kGT / W;
    S old[R];
    int64_t src[R], dst[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int orow = row0 + q * W + warp;
        dst[q] = -1;
        if (orow < nout) {
            src[q] = DOWN ? (u.off + pos[u.off + k + orow]) * nrhs + col : (u.off + pos[u.off + orow]) * nrhs + col;
            dst[q] = DOWN ? src[q] : (u.dst + orow) * nrhs + col;
            old[q] = X[src[q]];
        }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
        if (dst[q] < 0) continue;
        const int i = q * W + warp;
        S v;
        if constexpr (W == 1) {
            v = tot[i];
        } else {
            v = zero<S>();
            for (int s2 = 0; s2 < nsum; ++s2) v = s2 == 0 ? Ps[i * kGT + lane] : v + Ps[(s2 * kGT + i) * kGT + lane];
        }
        X[dst[q]] = old[q] + v;
    }
}

// ---- reduction of near-field partial sums ------------------------------------------
// U[e] = sum of the entry's partial sums (slot * 32 + row), in a fixed order.
// A thread owns W consecutive right-hand sides of one entry (one 16-byte
// load per partial sum when W * sizeof(S) = 16) and issues the loads of up
// to four partial sums before adding them in order.
template <class S, int W>
__global__ void reduce_kernel(const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                              const S* __restrict__ part, S* __restrict__ U, int nrhs, int64_t n_tot) {
    struct alignas(W * sizeof(S)) Vec { S v[W]; };
    const int nq = nrhs / W;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_tot * nq) return;
    const int64_t e = g / nq;
    const int c = (int)(g % nq) * W;
    Vec s;
#pragma unroll
    for (int w = 0; w < W; ++w) s.v[w] = zero<S>();
    const int64_t p1 = ptr[e + 1];
    for (int64_t p = ptr[e]; p < p1; p += 4) {
        Vec v[4];
        const int m = (int)min((int64_t)4, p1 - p);
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (t < m) v[t] = *reinterpret_cast<const Vec*>(part + idx[p + t] * nrhs + c);
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (t < m)
#pragma unroll
                for (int w = 0; w < W; ++w) s.v[w] += v[t].v[w];
    }
    *reinterpret_cast<Vec*>(U + e * nrhs + c) = s;
}

// ---- near field ------------------------------------------------------------------------
constexpr int kNearWarps = 8;

template <class Real, bool CPLX>
struct NearArgs {
    using V4 = typename RealT<Real>::V4;
    using S = typename Scal<Real, CPLX>::T;
    const WorkItem* items;
    int64_t n_items;
    const int64_t* box_off;
    const int32_t* box_n;
    const int32_t* box_nslot;
    const int32_t* slot_start;
    const int64_t* task_src;
    const uint64_t* task_mask;
    const int32_t* task_flags;
    const V4* X;
    const V4* Xlo;
    const S* Q;
    S* partial;
    int nrhs;
    Real kappa;
    Real kappa_lo;        // kappa - (Real)kappa: the FP32 2D Helmholtz phase uses both
};

__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float log_(float x) { return logf(x); }
__device__ __forceinline__ double log_(double x) { return log(x); }
__device__ __forceinline__ void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float j0_(float x) { return j0f(x); }
__device__ __forceinline__ double j0_(double x) { return j0(x); }
__device__ __forceinline__ float y0_(float x) { return y0f(x); }
__device__ __forceinline__ double y0_(double x) { return y0(x); }

// kernels with complex values: 3D and 2D Helmholtz
__host__ __device__ constexpr bool cplx_kind(int kind) { return kind == 2 || kind == 3; }

// kernel value without its constant factor (applied once per target):
// Laplace 2D: log r^2 (factor -1/(4 pi)); Laplace 3D: 1/r (factor 1/(4 pi));
// Helmholtz 3D: e^{i kappa r}/r (factor 1/(4 pi)).
template <class Real, int KIND> struct Green {
    using G = Real;
    static __device__ __forceinline__ Real eval(Real r2, Real) {
        return KIND == 0 ? log_(r2) : rsqrt_(r2);
    }
    static __device__ __forceinline__ Real zero_() { return Real(0); }
};
template <class Real> struct Green<Real, 2> {
    using G = Cx<Real>;
    static __device__ __forceinline__ Cx<Real> eval(Real r2, Real kappa) {
        const Real ri = rsqrt_(r2);
        Real s, c;
        sincos_(kappa * (r2 * ri), &s, &c);
        return {c * ri, s * ri};
    }
    static __device__ __forceinline__ Cx<Real> zero_() { return {Real(0), Real(0)}; }
};
// 2D Helmholtz: (i/4) H_0^(1)(kappa r) = (i/4) (J_0 + i Y_0); the 1/4 is in
// green_scale, the CUDA math library's Bessel functions give J_0 and Y_0
template <class Real> struct Green<Real, 3> {
    using G = Cx<Real>;
    static __device__ __forceinline__ Cx<Real> eval(Real r2, Real kappa) {
        const Real kr = kappa * sqrt(r2);
        return {-y0_(kr), j0_(kr)};
    }
    static __device__ __forceinline__ Cx<Real> zero_() { return {Real(0), Real(0)}; }
};
// ---- 2D Helmholtz in FP32 ---------------------------------------------------------------
// FP32 cannot carry the phase kappa r of a far pair: one ulp of r is 6e-8 r,
// so at kappa r ~ 100 the phase, and with it the kernel value, would be off by
// ~1e-5. The FP32 path therefore forms the coordinate differences from the hi
// and lo parts and the distance r = sqrt(dx^2 + dy^2) as double-float values
// (an unevaluated sum h + l; Knuth's two-sum, FMA-exact products, one Newton
// correction of the square root), and evaluates G without its factor 1/4:
//   x = kappa r < 8:  (-Y_0(x), J_0(x)) from the CUDA math library's y0f /
//                     j0f (at most 9 ulp on this range);
//   x >= 8:           Hankel's asymptotic expansion (Abramowitz & Stegun
//                     9.2.5, 9.2.9, 9.2.10) H_0^(1)(x) = sqrt(2 / (pi x))
//                     (P(x) + i Q(x)) e^{i (x - pi/4)}, with
//                     P = sum_k (-1)^k t_{2k} u^{2k}, Q = sum_k (-1)^{k+1}
//                     t_{2k+1} u^{2k+1}, u = 1 / (2x), t_0 = 1,
//                     t_m = t_{m-1} (2m - 1)^2 / (4m); six terms of each stay
//                     within 4e-8 of |H_0^(1)| for x >= 8. The phase x - pi/4
//                     is reduced modulo pi/2 by Cody and Waite's method (pi/2
//                     as a sum of three floats) in double-float arithmetic.
struct F2 {
    float h, l;
};
__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ F2 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, fmaf(a, b, -p)};
}
// (th + tl) - (sh + sl) as a double-float
__device__ __forceinline__ F2 df_diff(float th, float sh, float tl, float sl) {
    const F2 d = two_sum(th, -sh);
    return two_sum(d.h, __fadd_rn(d.l, __fsub_rn(tl, sl)));
}
__host__ __device__ constexpr double hankel_t(int m) {
    double v = 1.0;
    for (int j = 1; j <= m; ++j) v *= (double)((2 * j - 1) * (2 * j - 1)) / (4.0 * j);
    return v;
}
__device__ __forceinline__ Cx<float> helmholtz2d_f32(F2 dx, F2 dy, float kh, float kl) {
    // r^2 and r as double-floats
    const F2 px = two_prod(dx.h, dx.h), py = two_prod(dy.h, dy.h);
    const F2 s = two_sum(px.h, py.h);
    const float lo = s.l + px.l + py.l + 2.f * (dx.h * dx.l + dy.h * dy.l);
    const F2 r2 = two_sum(s.h, lo);
    if (!(r2.h > 0.f)) return {0.f, 0.f};
    const float rh = sqrtf(r2.h);
    const float rl = (fmaf(-rh, rh, r2.h) + r2.l) * (0.5f / rh);
    F2 x = two_prod(kh, rh);
    x.l += kh * rl + kl * rh;
    if (x.h < 8.f) return {-y0f(x.h), j0f(x.h)};
    constexpr double kPi = 3.14159265358979323846;
    const float u = 0.5f / x.h, v = u * u;
    const float P = 1.f + v * (-(float)hankel_t(2) + v * ((float)hankel_t(4) + v * (-(float)hankel_t(6) +
                    v * ((float)hankel_t(8) + v * (-(float)hankel_t(10))))));
    const float Q = u * (-(float)hankel_t(1) + v * ((float)hankel_t(3) + v * (-(float)hankel_t(5) +
                    v * ((float)hankel_t(7) + v * (-(float)hankel_t(9) + v * (float)hankel_t(11))))));
    const float amp = (float)0.79788456080286535588 * rsqrtf(x.h);     // sqrt(2 / pi) / sqrt(x)
    // chi = x - pi/4 = w + n pi/2, |w| <= pi/4 (plus rounding)
    constexpr float kP4h = (float)(kPi / 4);
    constexpr float kP4l = (float)(kPi / 4 - (double)(float)(kPi / 4));
    constexpr float kC1 = 1.5703125f;                                   // 8 significant bits: n C1 is exact
    constexpr float kC2 = (float)(kPi / 2 - 1.5703125);
    constexpr float kC3 = (float)(kPi / 2 - 1.5703125 - (double)(float)(kPi / 2 - 1.5703125));
    const F2 z = two_sum(x.h, -kP4h);
    const float zl = z.l + (x.l - kP4l);
    const float n = rintf(z.h * (float)(2.0 / kPi));
    float w = fmaf(-n, kC1, z.h);
    w = fmaf(-n, kC2, w);
    w = fmaf(-n, kC3, w);
    w += zl;
    float sw, cw;
    sincosf(w, &sw, &cw);
    const int qd = (int)n & 3;
    const float sc = qd == 0 ? sw : qd == 1 ? cw : qd == 2 ? -sw : -cw;     // sin chi
    const float cc = qd == 0 ? cw : qd == 1 ? -sw : qd == 2 ? -cw : sw;     // cos chi
    const float J = amp * (P * cc - Q * sc), Y = amp * (P * sc + Q * cc);
    return {-Y, J};
}

template <class G, class S> __device__ __forceinline__ void madd(S& acc, G g, S q);
template <> __device__ __forceinline__ void madd<float, float>(float& a, float g, float q) { a = fmaf(g, q, a); }
template <> __device__ __forceinline__ void madd<double, double>(double& a, double g, double q) { a = fma(g, q, a); }
template <> __device__ __forceinline__ void madd<Cx<float>, Cx<float>>(Cx<float>& a, Cx<float> g, Cx<float> q) {
    a.x = fmaf(g.x, q.x, a.x); a.x = fmaf(-g.y, q.y, a.x);
    a.y = fmaf(g.x, q.y, a.y); a.y = fmaf(g.y, q.x, a.y);
}
template <> __device__ __forceinline__ void madd<Cx<double>, Cx<double>>(Cx<double>& a, Cx<double> g, Cx<double> q) {
    a.x = fma(g.x, q.x, a.x); a.x = fma(-g.y, q.y, a.x);
    a.y = fma(g.x, q.y, a.y); a.y = fma(g.y, q.x, a.y);
}

template <int KIND> __host__ __device__ constexpr double green_scale() {
    return KIND == 0   ? -1.0 / (4.0 * 3.14159265358979323846)
           : KIND == 3 ? 0.25
                       : 1.0 / (4.0 * 3.14159265358979323846);
}

// One source slot [s0, s1) against the warp's 32 targets.
template <class Real, int KIND, int RT, bool ADJ>
__device__ __forceinline__ void near_slot(const NearArgs<Real, cplx_kind(KIND)>& a, int64_t s0, int64_t s1, int r0,
                                          typename RealT<Real>::V4 tx, typename RealT<Real>::V4 tl,
                                          typename RealT<Real>::V4* sx, typename RealT<Real>::V4* sl,
                                          typename Scal<Real, cplx_kind(KIND)>::T* sq, int lane,
                                          typename Scal<Real, cplx_kind(KIND)>::T* part) {
    using S = typename Scal<Real, cplx_kind(KIND)>::T;
    using Gr = Green<Real, KIND>;
    // FP32 lo parts: touching leaves (arbitrarily close pairs), and every pair
    // of the 2D Helmholtz kernel (its phase needs the distance to ~1e-9)
    constexpr bool H2F = KIND == 3 && sizeof(Real) == 4;
    constexpr bool LO = (ADJ || H2F) && sizeof(Real) == 4;
    for (int64_t b = s0; b < s1; b += 32) {
        const int cnt = (int)min((int64_t)32, s1 - b);
        if (lane < cnt) {
            sx[lane] = a.X[b + lane];
            if (LO) sl[lane] = a.Xlo[b + lane];
#pragma unroll
            for (int r = 0; r < RT; ++r)
                sq[lane * RT + r] = (r0 + r < a.nrhs) ? a.Q[(b + lane) * a.nrhs + r0 + r] : zero<S>();
        }
        __syncwarp();
        for (int j = 0; j < cnt; ++j) {
            const typename RealT<Real>::V4 s = sx[j];
            typename Gr::G g;
            if constexpr (H2F) {
                const typename RealT<Real>::V4 l = sl[j];
                g = helmholtz2d_f32(df_diff(tx.x, s.x, tl.x, l.x), df_diff(tx.y, s.y, tl.y, l.y), a.kappa,
                                    a.kappa_lo);
            } else {
                Real dx = tx.x - s.x, dy = tx.y - s.y, dz = tx.z - s.z;
                if (LO) {
                    const typename RealT<Real>::V4 l = sl[j];
                    dx += tl.x - l.x;
                    dy += tl.y - l.y;
                    dz += tl.z - l.z;
                }
                const Real r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                g = Gr::eval(r2, a.kappa);
                if (ADJ && !(r2 > Real(0))) g = Gr::zero_();
            }
#pragma unroll
            for (int r = 0; r < RT; ++r) madd(part[r], g, sq[j * RT + r]);
        }
        __syncwarp();
    }
}

template <class Real, int KIND, int RT>
__global__ void __launch_bounds__(kNearWarps * 32) near_kernel(const NearArgs<Real, cplx_kind(KIND)> a, int r0) {
    using V4 = typename RealT<Real>::V4;
    using S = typename Scal<Real, cplx_kind(KIND)>::T;
    __shared__ V4 s_x[kNearWarps][32];
    __shared__ V4 s_l[kNearWarps][sizeof(Real) == 4 ? 32 : 1];
    __shared__ S s_q[kNearWarps][32 * RT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item_id = (int64_t)blockIdx.x * kNearWarps + warp;
    if (item_id >= a.n_items) return;
    const WorkItem it = a.items[item_id];
    const int64_t B = it.tgt_box;
    const int64_t boff = a.box_off[B];
    const int t = it.t0 + lane;
    const bool valid = t < a.box_n[B];
    const int32_t* ssB = a.slot_start + B * (kMaxSlots + 1);
    int myslot = 0;
    for (int c = 1; c < a.box_nslot[B]; ++c)
        if (t >= ssB[c]) myslot = c;
    V4 tx = {0, 0, 0, 0}, tl = {0, 0, 0, 0};
    if (valid) {
        tx = a.X[boff + t];
        if (sizeof(Real) == 4) tl = a.Xlo[boff + t];
    }
    S acc[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) acc[r] = zero<S>();
    for (int tk = it.task_lo; tk < it.task_hi; ++tk) {
        const int64_t src = a.task_src[tk];
        const unsigned row = (unsigned)(a.task_mask[tk] >> (myslot * 8)) & 0xffu;
        const bool adj = (a.task_flags[tk] & TASK_ADJ) != 0;
        const int64_t soff = a.box_off[src];
        const int nsl = a.box_nslot[src];
        const int32_t* ssS = a.slot_start + src * (kMaxSlots + 1);
        for (int c = 0; c < nsl; ++c) {
            const bool skip = !valid || ((row >> c) & 1u);
            if (__all_sync(0xffffffffu, skip)) continue;
            S part[RT];
#pragma unroll
            for (int r = 0; r < RT; ++r) part[r] = zero<S>();
            if (adj)
                near_slot<Real, KIND, RT, true>(a, soff + ssS[c], soff + ssS[c + 1], r0, tx, tl, s_x[warp],
                                                s_l[warp], s_q[warp], lane, part);
            else
                near_slot<Real, KIND, RT, false>(a, soff + ssS[c], soff + ssS[c + 1], r0, tx, tl, s_x[warp],
                                                 s_l[warp], s_q[warp], lane, part);
            if (!skip) {
#pragma unroll
                for (int r = 0; r < RT; ++r) acc[r] += part[r];
            }
        }
    }
    const Real scale = (Real)green_scale<KIND>();
#pragma unroll
    for (int r = 0; r < RT; ++r)
        if (r0 + r < a.nrhs) a.partial[(item_id * kChunk + lane) * a.nrhs + r0 + r] = scale * acc[r];
}

// returns the number of launches; right-hand sides go in passes of 8 (a
// single 32-wide pass measured slower: its registers and shared memory halve
// the resident warps)
template <class Real, int KIND>
int launch_near_kind(const NearArgs<Real, cplx_kind(KIND)>& a, int nrhs, unsigned grid, cudaStream_t st) {
    if (nrhs == 1) {
        near_kernel<Real, KIND, 1><<<grid, kNearWarps * 32, 0, st>>>(a, 0);
        return 1;
    }
    constexpr int RT = 8;
    int n = 0;
    for (int r0 = 0; r0 < nrhs; r0 += RT, ++n) near_kernel<Real, KIND, RT><<<grid, kNearWarps * 32, 0, st>>>(a, r0);
    return n;
}

template <class Real, bool CPLX>
int launch_near(int kind, const NearArgs<Real, CPLX>& a, int nrhs, unsigned grid, cudaStream_t st);
template <>
inline int launch_near<float, false>(int kind, const NearArgs<float, false>& a, int nrhs, unsigned grid,
                                      cudaStream_t st) {
    return kind == 0 ? launch_near_kind<float, 0>(a, nrhs, grid, st) : launch_near_kind<float, 1>(a, nrhs, grid, st);
}
template <>
inline int launch_near<double, false>(int kind, const NearArgs<double, false>& a, int nrhs, unsigned grid,
                                       cudaStream_t st) {
    return kind == 0 ? launch_near_kind<double, 0>(a, nrhs, grid, st)
                     : launch_near_kind<double, 1>(a, nrhs, grid, st);
}
template <>
inline int launch_near<float, true>(int kind, const NearArgs<float, true>& a, int nrhs, unsigned grid,
                                     cudaStream_t st) {
    return kind == 3 ? launch_near_kind<float, 3>(a, nrhs, grid, st) : launch_near_kind<float, 2>(a, nrhs, grid, st);
}
template <>
inline int launch_near<double, true>(int kind, const NearArgs<double, true>& a, int nrhs, unsigned grid,
                                      cudaStream_t st) {
    return kind == 3 ? launch_near_kind<double, 3>(a, nrhs, grid, st)
                     : launch_near_kind<double, 2>(a, nrhs, grid, st);
}

}  // namespace skel
