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
template <class S>
__global__ void permute_in(const int64_t* __restrict__ pe, const int64_t* __restrict__ pp,
                           const S* __restrict__ q, S* __restrict__ Q, int64_t N, int nrhs) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N * nrhs) return;
    const int64_t i = g % N, r = g / N;
    Q[pe[i] * nrhs + r] = q[r * N + pp[i]];
}

template <class S>
__global__ void permute_out(const int64_t* __restrict__ pe, const int64_t* __restrict__ pp,
                            const S* __restrict__ U, S* __restrict__ u, int64_t N, int nrhs) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N * nrhs) return;
    const int64_t i = g % N, r = g / N;
    u[r * N + pp[i]] = U[pe[i] * nrhs + r];
}

// ---- upward: qhat_S = q_S + T q_R into the parent's slot ---------------------------
// One CTA per box, a small GEMM (k x r) x (r x nrhs): rows of q_R are gathered
// into shared memory 32 at a time; each thread owns up to kOwn (row, group of
// RG right-hand sides) outputs; T (column-major, k contiguous) is read
// coalesced across rows.
constexpr int kUpThreads = 256;
constexpr int kOwn = 4;
constexpr int kJT = 32;

template <class S, int RG>
__global__ void __launch_bounds__(kUpThreads) up_kernel(const UpBox* __restrict__ up, const int32_t* __restrict__ pos,
                                                        const S* __restrict__ T, S* Q, int nrhs, bool conjT) {
    extern __shared__ unsigned char smem_raw[];
    S* qs = reinterpret_cast<S*>(smem_raw);              // kJT x nrhs
    const UpBox u = up[blockIdx.x];
    const int k = u.k, r = u.n - u.k;
    const int ng = (nrhs + RG - 1) / RG;
    const int total = k * ng;
    for (int base = 0; base < total; base += kUpThreads * kOwn) {
        S acc[kOwn][RG];
#pragma unroll
        for (int o = 0; o < kOwn; ++o)
#pragma unroll
            for (int c = 0; c < RG; ++c) acc[o][c] = zero<S>();
        for (int j0 = 0; j0 < r; j0 += kJT) {
            const int jn = min(kJT, r - j0);
            __syncthreads();
            for (int e = threadIdx.x; e < jn * nrhs; e += kUpThreads) {
                const int jj = e / nrhs, c = e % nrhs;
                qs[e] = Q[(u.off + pos[u.off + k + j0 + jj]) * nrhs + c];
            }
            __syncthreads();
#pragma unroll
            for (int o = 0; o < kOwn; ++o) {
                const int task = base + o * kUpThreads + threadIdx.x;
                if (task >= total) break;
                const int i = task % k, g = task / k;
                const S* Ti = T + u.T_off + i + (int64_t)j0 * k;
                for (int jj = 0; jj < jn; ++jj) {
                    S tv = Ti[(int64_t)jj * k];
                    if (conjT) tv = conj(tv);
#pragma unroll
                    for (int c = 0; c < RG; ++c)
                        if (g * RG + c < nrhs) acc[o][c] += tv * qs[jj * nrhs + g * RG + c];
                }
            }
        }
#pragma unroll
        for (int o = 0; o < kOwn; ++o) {
            const int task = base + o * kUpThreads + threadIdx.x;
            if (task >= total) break;
            const int i = task % k, g = task / k;
            const int64_t src = (u.off + pos[u.off + i]) * nrhs, dst = (u.dst + i) * nrhs;
#pragma unroll
            for (int c = 0; c < RG; ++c) {
                const int cc = g * RG + c;
                if (cc < nrhs) Q[dst + cc] = Q[src + cc] + acc[o][c];
            }
        }
    }
}

// ---- downward: uhat = U[parent slot]; u_S += uhat; u_R += T^* uhat -------------------
// One CTA per box; uhat rows are staged in shared memory 32 at a time and the
// transposed copy Tt (r x k, column-major: r contiguous) is read coalesced
// across the output rows j of R.
template <class S, int RG>
__global__ void __launch_bounds__(kUpThreads) down_kernel(const UpBox* __restrict__ up, const int32_t* __restrict__ pos,
                                                          const S* __restrict__ Tt, S* U, int nrhs, bool transpose) {
    extern __shared__ unsigned char smem_raw[];
    S* us = reinterpret_cast<S*>(smem_raw);              // kJT x nrhs
    const UpBox u = up[blockIdx.x];
    const int k = u.k, r = u.n - u.k;
    for (int e = threadIdx.x; e < k * nrhs; e += kUpThreads) {
        const int i = e / nrhs, c = e % nrhs;
        U[(u.off + pos[u.off + i]) * nrhs + c] += U[(u.dst + i) * nrhs + c];
    }
    const int ng = (nrhs + RG - 1) / RG;
    const int total = r * ng;
    for (int base = 0; base < total; base += kUpThreads * kOwn) {
        S acc[kOwn][RG];
#pragma unroll
        for (int o = 0; o < kOwn; ++o)
#pragma unroll
            for (int c = 0; c < RG; ++c) acc[o][c] = zero<S>();
        for (int i0 = 0; i0 < k; i0 += kJT) {
            const int in = min(kJT, k - i0);
            __syncthreads();
            for (int e = threadIdx.x; e < in * nrhs; e += kUpThreads) us[e] = U[(u.dst + i0) * nrhs + e];
            __syncthreads();
#pragma unroll
            for (int o = 0; o < kOwn; ++o) {
                const int task = base + o * kUpThreads + threadIdx.x;
                if (task >= total) break;
                const int j = task % r, g = task / r;
                const S* Tj = Tt + u.T_off + j + (int64_t)i0 * r;
                for (int ii = 0; ii < in; ++ii) {
                    S tv = Tj[(int64_t)ii * r];
                    if (!transpose) tv = conj(tv);
#pragma unroll
                    for (int c = 0; c < RG; ++c)
                        if (g * RG + c < nrhs) acc[o][c] += tv * us[ii * nrhs + g * RG + c];
                }
            }
        }
#pragma unroll
        for (int o = 0; o < kOwn; ++o) {
            const int task = base + o * kUpThreads + threadIdx.x;
            if (task >= total) break;
            const int j = task % r, g = task / r;
            const int64_t e = (u.off + pos[u.off + k + j]) * nrhs;
#pragma unroll
            for (int c = 0; c < RG; ++c) {
                const int cc = g * RG + c;
                if (cc < nrhs) U[e + cc] += acc[o][c];
            }
        }
    }
}

// ---- reduction of near-field partial sums ------------------------------------------
// U[e] = sum of the entry's partial sums (slot * 32 + row), in a fixed order
template <class S>
__global__ void reduce_kernel(const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                              const S* __restrict__ part, S* __restrict__ U, int nrhs, int64_t n_tot) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_tot * nrhs) return;
    const int64_t e = g / nrhs;
    const int r = (int)(g % nrhs);
    S s = zero<S>();
    for (int64_t p = ptr[e]; p < ptr[e + 1]; ++p) s += part[idx[p] * nrhs + r];
    U[e * nrhs + r] = s;
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
};

__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float log_(float x) { return logf(x); }
__device__ __forceinline__ double log_(double x) { return log(x); }
__device__ __forceinline__ void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_(double x, double* s, double* c) { sincos(x, s, c); }

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
    return KIND == 0 ? -1.0 / (4.0 * 3.14159265358979323846) : 1.0 / (4.0 * 3.14159265358979323846);
}

// One source slot [s0, s1) against the warp's 32 targets.
template <class Real, int KIND, int RT, bool ADJ>
__device__ __forceinline__ void near_slot(const NearArgs<Real, KIND == 2>& a, int64_t s0, int64_t s1, int r0,
                                          typename RealT<Real>::V4 tx, typename RealT<Real>::V4 tl,
                                          typename RealT<Real>::V4* sx, typename RealT<Real>::V4* sl,
                                          typename Scal<Real, KIND == 2>::T* sq, int lane,
                                          typename Scal<Real, KIND == 2>::T* part) {
    using S = typename Scal<Real, KIND == 2>::T;
    using Gr = Green<Real, KIND>;
    constexpr bool LO = ADJ && sizeof(Real) == 4;
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
            Real dx = tx.x - s.x, dy = tx.y - s.y, dz = tx.z - s.z;
            if (LO) {
                const typename RealT<Real>::V4 l = sl[j];
                dx += tl.x - l.x;
                dy += tl.y - l.y;
                dz += tl.z - l.z;
            }
            const Real r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            typename Gr::G g = Gr::eval(r2, a.kappa);
            if (ADJ && !(r2 > Real(0))) g = Gr::zero_();
#pragma unroll
            for (int r = 0; r < RT; ++r) madd(part[r], g, sq[j * RT + r]);
        }
        __syncwarp();
    }
}

template <class Real, int KIND, int RT>
__global__ void __launch_bounds__(kNearWarps * 32) near_kernel(const NearArgs<Real, KIND == 2> a, int r0) {
    using V4 = typename RealT<Real>::V4;
    using S = typename Scal<Real, KIND == 2>::T;
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
int launch_near_kind(const NearArgs<Real, KIND == 2>& a, int nrhs, unsigned grid, cudaStream_t st) {
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
inline int launch_near<float, true>(int, const NearArgs<float, true>& a, int nrhs, unsigned grid,
                                     cudaStream_t st) {
    return launch_near_kind<float, 2>(a, nrhs, grid, st);
}
template <>
inline int launch_near<double, true>(int, const NearArgs<double, true>& a, int nrhs, unsigned grid,
                                      cudaStream_t st) {
    return launch_near_kind<double, 2>(a, nrhs, grid, st);
}

}  // namespace skel
