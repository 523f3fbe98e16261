// Algorithm 2 (FMM apply) on the GPU, and the device plan around it.
//
// One apply, all on one stream:
//   permute_in            q (user order)  -> leaf entries of Q
//   updown_kernel (up),   qhat_S = q_S + T q_R, written into the parent's slot
//     l = L..2
//   translations          every translation (ifo / ifs / tfo / level-1 sum,
//                         subtractions folded in as slot masks, see layout.cpp):
//                         FP64 / FP32 / complex: near_kernel into per-work-item
//                         partial sums, then reduce_kernel -> U (fixed order);
//                         FP32_TC: tc_bprep_kernel + tc_near_kernel (kernel
//                         evaluated on the fly) or tc_stored_kernel (stored
//                         tiles) per 32 right-hand sides, writing U directly
//   updown_kernel (down), uhat_S = U[parent slot]; u_S += uhat; u_R += T^* uhat
//     l = 2..L
//   permute_out           leaf entries of U -> u (user order)
//
// device_autotune measures the variants (up/down kernel per level; stored or
// on-the-fly tiles) on a plan and keeps the faster ones.
//
// The CUDA-core near field: a warp owns 32 targets (one per lane, in
// registers) and streams the sources of its task range through a per-warp
// shared-memory tile, every lane reading the same source (a broadcast).
// Tasks between touching leaves (TASK_ADJ) hold the only close pairs: in FP32
// they difference coordinates split into hi + lo floats, so a pair at
// distance r keeps ~1e-7 relative accuracy however small r is, and they test
// r^2 > 0 (the zero diagonal); every other task has pairs at least one small
// box apart and uses the hi part alone.
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>

#include "device.h"
#include "skel_kernels.cuh"
#include "tc_kernels.cuh"
#include "tc_complex.cuh"
#include "tc_stored_ring.cuh"
#include "tc_updown.cuh"
#include "updown_async.cuh"

namespace skel {

#define CUDA_CHECK(x)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (x);                                                           \
        if (e_ != cudaSuccess)                                                          \
            throw Error(-3, std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x); \
    } while (0)

struct DeviceBuffers {
    void* X = nullptr;       // Real4 per entry: (x, y, z, 0); FP32: hi part
    void* Xlo = nullptr;     // FP32 only: lo part
    void* T = nullptr;       // Real or complex, per box k x r column-major
    void* Tt = nullptr;      // the same blocks transposed (r x k column-major)
    void* Q = nullptr;       // n_tot * nrhs_max
    void* U = nullptr;
    void* partial = nullptr; // n_items * 32 * nrhs_max
};

namespace {
std::atomic<int> g_fail_countdown{0};
}  // namespace

void set_alloc_failure(int countdown) { g_fail_countdown.store(countdown > 0 ? countdown : 0); }

bool alloc_should_fail() {
    int c = g_fail_countdown.load();
    while (c > 0) {
        if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
    }
    return false;
}

namespace {

// NVTX range around a phase of the apply (host side; visible to nsys and ncu)
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

template <class T>
T* dalloc(size_t n, int64_t& bytes) {
    void* p = nullptr;
    if (n == 0) n = 1;
    if (alloc_should_fail()) throw Error(-2, "cudaMalloc failed: simulated allocation failure (test hook)");
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(-2, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    bytes += (int64_t)(n * sizeof(T));
    return (T*)p;
}

template <class T>
T* upload(const std::vector<T>& v, int64_t& bytes) {
    T* p = dalloc<T>(v.size(), bytes);
    if (!v.empty()) CUDA_CHECK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}

template <class Real>
void make_buffers(DevicePlan* dp, const Layout& lay, DeviceBuffers* b) {
    using V = typename RealT<Real>::V4;
    const int64_t nt = lay.n_tot;
    const int w = dp->cplx ? 2 : 1;
    std::vector<V> xh(nt), xl(nt);
    for (int64_t e = 0; e < nt; ++e) {
        double x[4] = {lay.X[e * 4], lay.X[e * 4 + 1], lay.X[e * 4 + 2], 0.0};
        Real h[4], l[4];
        for (int d = 0; d < 4; ++d) {
            h[d] = (Real)x[d];
            l[d] = (Real)(x[d] - (double)h[d]);
        }
        xh[e] = V{h[0], h[1], h[2], h[3]};
        xl[e] = V{l[0], l[1], l[2], l[3]};
    }
    b->X = upload(xh, dp->bytes);
    if (sizeof(Real) == 4) b->Xlo = upload(xl, dp->bytes);
    std::vector<Real> tr(lay.T.size()), tt(lay.T.size());
    for (size_t i = 0; i < lay.T.size(); ++i) tr[i] = (Real)lay.T[i];
    for (const UpBox& u : lay.up) {
        const int k = u.k, r = u.n - u.k;
        for (int j = 0; j < r; ++j)
            for (int i = 0; i < k; ++i)
                for (int c = 0; c < w; ++c)
                    tt[(u.T_off + j + (int64_t)i * r) * w + c] = tr[(u.T_off + i + (int64_t)j * k) * w + c];
    }
    b->T = upload(tr, dp->bytes);
    b->Tt = upload(tt, dp->bytes);
    b->Q = dalloc<Real>((size_t)nt * dp->nrhs_max * w, dp->bytes);
    b->U = dalloc<Real>((size_t)nt * dp->nrhs_max * w, dp->bytes);
    const int64_t slots = std::max<int64_t>(dp->n_items, sizeof(Real) == 4 ? dp->tc_n_slots : 0);
    b->partial = dalloc<Real>((size_t)slots * kChunk * dp->nrhs_max * w, dp->bytes);
}

void free_buffers(DeviceBuffers* b) {
    if (!b) return;
    cudaFree(b->X);
    cudaFree(b->Xlo);
    cudaFree(b->T);
    cudaFree(b->Tt);
    cudaFree(b->Q);
    cudaFree(b->U);
    cudaFree(b->partial);
    delete b;
}

inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// warps per CTA of the up/down kernel for a level whose inner index has nch
// chunks of 32: the default rule (one warp per chunk, at most 4)
inline int ud_default_warps(int nch) { return nch >= 4 ? 4 : nch >= 2 ? 2 : 1; }

template <class S, bool DOWN, int W>
void ud_launch(dim3 grid, const UpBox* up, const int32_t* pos, const S* T, S* X, int nrhs, bool conj_op,
               cudaStream_t st) {
    if constexpr (W <= ud_streams<S>())
        updown_kernel<S, DOWN, W><<<grid, 32 * W, ud_smem<S>(W), st>>>(up, pos, T, X, nrhs, conj_op);
    else
        throw Error(-1, "up/down: more warps than streams");
}

template <class S, bool DOWN>
void ud_set_attributes() {
    CUDA_CHECK(cudaFuncSetAttribute(updown_kernel<S, DOWN, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUdSmemMax));
    CUDA_CHECK(cudaFuncSetAttribute(updown_kernel<S, DOWN, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUdSmemMax));
    if constexpr (ud_streams<S>() >= 4)
        CUDA_CHECK(cudaFuncSetAttribute(updown_kernel<S, DOWN, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUdSmemMax));
    if constexpr (ud_streams<S>() >= 8)
        CUDA_CHECK(cudaFuncSetAttribute(updown_kernel<S, DOWN, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUdSmemMax));
}

template <class S>
void ud_attributes_once() {
    static bool done = false;
    if (done) return;
    ud_set_attributes<S, false>();
    ud_set_attributes<S, true>();
    if constexpr (std::is_same<S, float>::value) {
        CUDA_CHECK(cudaFuncSetAttribute(updown_rows_kernel<false, 4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ud_rows_smem(4)));
        CUDA_CHECK(cudaFuncSetAttribute(updown_rows_kernel<true, 4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ud_rows_smem(4)));
        CUDA_CHECK(cudaFuncSetAttribute(updown_rows_kernel<false, 8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ud_rows_smem(8)));
        CUDA_CHECK(cudaFuncSetAttribute(updown_rows_kernel<true, 8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ud_rows_smem(8)));
        CUDA_CHECK(cudaFuncSetAttribute(updown_rows_kernel<false, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ud_rows_smem(4)));
        CUDA_CHECK(cudaFuncSetAttribute(updown_rows_kernel<true, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ud_rows_smem(4)));
        CUDA_CHECK(cudaFuncSetAttribute(updown_rows_kernel<false, 8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ud_rows_smem(8)));
        CUDA_CHECK(cudaFuncSetAttribute(updown_rows_kernel<true, 8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ud_rows_smem(8)));
    }
    done = true;
}

// launch-shape codes of the FP32 up/down passes: 1, 2, 4, 8 = updown_kernel
// with that many warps per CTA (one 32-row block); kUdAsync + NW =
// updown_rows_kernel with NW warps owning 32 NW rows (same result bit for bit)
constexpr int kUdAsync = 16;

template <bool DOWN, int NW>
void ud_rows_launch(const DevicePlan* dp, int l, int nrhs, const float* T, float* X, cudaStream_t st) {
    constexpr int wi = NW == 1 ? 0 : NW == 2 ? 1 : NW == 4 ? 2 : 3;
    const std::vector<int64_t>& ptr = dp->ud_work_ptr[DOWN ? 1 : 0][wi];
    const int64_t w0 = ptr[l], w1 = ptr[l + 1];
    if (w1 <= w0) return;
    const dim3 grid((unsigned)(w1 - w0), 1, ceil_div(nrhs, kGT));
    const int2* work = dp->ud_work[DOWN ? 1 : 0][wi] + w0;
    if (nrhs % 4 == 0 && dp->ud_tp) {
        const float* Tp = DOWN ? dp->ud_ttp : dp->ud_tp;
        const int64_t* off = DOWN ? dp->ud_ttp_off : dp->ud_tp_off;
        updown_rows_kernel<DOWN, NW, true><<<grid, 32 * NW, ud_rows_smem(NW), st>>>(dp->up, work, dp->pos, Tp, off, X,
                                                                                     nrhs);
    } else {
        updown_rows_kernel<DOWN, NW, false><<<grid, 32 * NW, ud_rows_smem(NW), st>>>(dp->up, work, dp->pos, T, nullptr,
                                                                                      X, nrhs);
    }
}

// one level of the upward or downward pass on the tensor cores (FP32_TC,
// real kernels): one launch per 32 right-hand sides; returns the launches
int up_down_tc(bool down, DevicePlan* dp, int l, float* X, int nrhs, cudaStream_t st) {
    static std::atomic<bool> attr{false};
    if (!attr.exchange(true)) {
        CUDA_CHECK(cudaFuncSetAttribute(tc_ud_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUdSmemRequest));
        CUDA_CHECK(cudaFuncSetAttribute(tc_ud_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUdSmemRequest));
    }
    const std::vector<int64_t>& ptr = down ? dp->ud_ptr_down : dp->ud_ptr_up;
    const int64_t i0 = ptr[l], i1 = ptr[l + 1];
    if (i1 <= i0) return 0;
    UdArgs a;
    a.items = static_cast<const UdItem*>(down ? dp->ud_items_down : dp->ud_items_up) + i0;
    a.up = dp->up;
    a.pos = dp->pos;
    a.A = down ? dp->ud_a_down : dp->ud_a_up;
    a.X = X;
    a.n_tot = dp->n_tot;
    a.nrhs = nrhs;
    a.status = dp->status;
    a.wait_ns = kWaitLimitNs;
    int launches = 0;
    for (int r0 = 0; r0 < nrhs; r0 += kTcN, ++launches) {
        a.r0 = r0;
        if (down) tc_ud_kernel<true><<<(unsigned)(i1 - i0), kTcThreads, kUdSmemRequest, st>>>(a);
        else tc_ud_kernel<false><<<(unsigned)(i1 - i0), kTcThreads, kUdSmemRequest, st>>>(a);
        CUDA_CHECK(cudaGetLastError());
    }
    return launches;
}

// one level of the upward or downward pass; warps = 0: the level's setting
// (autotuned for FP32, else the default rule)
template <class S>
void up_down(bool down, const DevicePlan* dp, int l, const S* T, S* X, int nrhs, bool conj_op, cudaStream_t st,
             int warps = 0) {
    ud_attributes_once<S>();
    const int64_t b0 = dp->up_level_ptr[l], b1 = dp->up_level_ptr[l + 1];
    const int nout = down ? dp->up_level_maxr[l] : dp->up_level_maxk[l];
    const int ninner = down ? dp->up_level_maxk[l] : dp->up_level_maxr[l];
    const dim3 grid((unsigned)(b1 - b0), std::max(1u, ceil_div(nout, kGT)), ceil_div(nrhs, kGT));
    int W = warps;
    if (W == 0 && std::is_same<S, float>::value) {
        const std::vector<int8_t>& t = down ? dp->ud_warps_down : dp->ud_warps_up;
        if (l < (int)t.size() && t[l] > 0) W = t[l];
    }
    if (W == 0) W = ud_default_warps((ninner + kGT - 1) / kGT);
    const UpBox* up = dp->up + b0;
    if constexpr (std::is_same<S, float>::value) {
        if (W > kUdAsync) {
            switch (W - kUdAsync) {
                case 1: down ? ud_rows_launch<true, 1>(dp, l, nrhs, T, X, st)
                             : ud_rows_launch<false, 1>(dp, l, nrhs, T, X, st); break;
                case 2: down ? ud_rows_launch<true, 2>(dp, l, nrhs, T, X, st)
                             : ud_rows_launch<false, 2>(dp, l, nrhs, T, X, st); break;
                case 4: down ? ud_rows_launch<true, 4>(dp, l, nrhs, T, X, st)
                             : ud_rows_launch<false, 4>(dp, l, nrhs, T, X, st); break;
                default: down ? ud_rows_launch<true, 8>(dp, l, nrhs, T, X, st)
                              : ud_rows_launch<false, 8>(dp, l, nrhs, T, X, st); break;
            }
            return;
        }
    }
    W = std::min(W, ud_streams<S>());
    switch (W) {
        case 1: down ? ud_launch<S, true, 1>(grid, up, dp->pos, T, X, nrhs, conj_op, st)
                     : ud_launch<S, false, 1>(grid, up, dp->pos, T, X, nrhs, conj_op, st); break;
        case 2: down ? ud_launch<S, true, 2>(grid, up, dp->pos, T, X, nrhs, conj_op, st)
                     : ud_launch<S, false, 2>(grid, up, dp->pos, T, X, nrhs, conj_op, st); break;
        case 4: down ? ud_launch<S, true, 4>(grid, up, dp->pos, T, X, nrhs, conj_op, st)
                     : ud_launch<S, false, 4>(grid, up, dp->pos, T, X, nrhs, conj_op, st); break;
        default: down ? ud_launch<S, true, 8>(grid, up, dp->pos, T, X, nrhs, conj_op, st)
                      : ud_launch<S, false, 8>(grid, up, dp->pos, T, X, nrhs, conj_op, st); break;
    }
}

template <class S>
void reduce(const int64_t* ptr, const int64_t* idx, const S* part, S* U, int nrhs, int64_t n_tot, cudaStream_t st) {
    constexpr int W = 16 / sizeof(S);
    if (W > 1 && nrhs % W == 0) {
        const int64_t n = n_tot * (nrhs / W);
        reduce_kernel<S, W><<<ceil_div(n, 256), 256, 0, st>>>(ptr, idx, part, U, nrhs, n_tot);
    } else {
        const int64_t n = n_tot * nrhs;
        reduce_kernel<S, 1><<<ceil_div(n, 256), 256, 0, st>>>(ptr, idx, part, U, nrhs, n_tot);
    }
}

template <class S>
void permute(bool out, const DevicePlan* dp, const S* src, S* dst, int nrhs, cudaStream_t st) {
    const int64_t N = dp->N;
    if (nrhs >= 8) {
        const dim3 grid(ceil_div(N, kPermTile), ceil_div(nrhs, kPermTile));
        if (out) permute_out<S><<<grid, kPermThreads, 0, st>>>(dp->eop, dp->eop2, src, dst, N, nrhs);
        else permute_in<S><<<grid, kPermThreads, 0, st>>>(dp->eop, dp->eop2, src, dst, N, nrhs);
    } else {
        const int64_t n = N * nrhs;
        if (out) permute_out_narrow<S><<<ceil_div(n, 256), 256, 0, st>>>(dp->eop, dp->eop2, src, dst, N, nrhs);
        else permute_in_narrow<S><<<ceil_div(n, 256), 256, 0, st>>>(dp->eop, dp->eop2, src, dst, N, nrhs);
    }
}

constexpr int kProfEvents = 8;   // 7 phase boundaries + the start of the main translation kernel
constexpr int kMainEvent = 7;

inline void mark(DevicePlan* dp, int i, cudaStream_t st) {
    if (dp->prof_count < dp->prof_cap)
        CUDA_CHECK(cudaEventRecord((cudaEvent_t)dp->events[dp->prof_count * kProfEvents + i], st));
}

template <class Real, bool CPLX>
NearArgs<Real, CPLX> near_args(DevicePlan* dp, DeviceBuffers* b, const WorkItem* items, int64_t n_items, int nrhs) {
    NearArgs<Real, CPLX> a;
    a.items = items;
    a.n_items = n_items;
    a.box_off = dp->box_off;
    a.box_n = dp->box_n;
    a.box_nslot = dp->box_nslot;
    a.slot_start = dp->slot_start;
    a.task_src = dp->task_src;
    a.task_mask = dp->task_mask;
    a.task_flags = dp->task_flags;
    a.X = (const typename RealT<Real>::V4*)b->X;
    a.Xlo = (const typename RealT<Real>::V4*)b->Xlo;
    a.Q = (const typename Scal<Real, CPLX>::T*)b->Q;
    a.partial = (typename Scal<Real, CPLX>::T*)b->partial;
    a.nrhs = nrhs;
    a.kappa = (Real)dp->kappa;
    a.kappa_lo = (Real)(dp->kappa - (double)(Real)dp->kappa);
    return a;
}

// tensor-core translations (real kernels, FP32): the CUDA-core items for
// the small non-leaf boxes and the reduction of their partial sums (which
// writes every row of U, zero where no CUDA-core item contributes), then one
// tensor-core pass per 32 right-hand sides, whose items write their rows of U
// directly (each row has exactly one item)
// dynamic shared memory above 48 KB for every tensor-core kernel (once per process)
void set_tc_attributes() {
    static bool done = false;
    if (done) return;
    CUDA_CHECK(cudaFuncSetAttribute(tc_near_kernel<0, kRecNone, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemRequest));
    CUDA_CHECK(cudaFuncSetAttribute(tc_near_kernel<1, kRecNone, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemRequest));
    CUDA_CHECK(cudaFuncSetAttribute(tc_near_kernel<0, kRecNone, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemRequest));
    CUDA_CHECK(cudaFuncSetAttribute(tc_near_kernel<1, kRecNone, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemRequest));
    CUDA_CHECK(cudaFuncSetAttribute(tc_near_kernel<0, kRecNone, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemRequest));
    CUDA_CHECK(cudaFuncSetAttribute(tc_near_kernel<1, kRecNone, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemRequest));
    CUDA_CHECK(cudaFuncSetAttribute(tc_near_kernel<0, kRecTiles>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemRequest));
    CUDA_CHECK(cudaFuncSetAttribute(tc_near_kernel<1, kRecTiles>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemRequest));
    CUDA_CHECK(cudaFuncSetAttribute(tc_near_kernel<0, kRecSym>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemRequest));
    CUDA_CHECK(cudaFuncSetAttribute(tc_near_kernel<1, kRecSym>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemRequest));
    CUDA_CHECK(cudaFuncSetAttribute(tc_stored_kernel<0, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, tcs_smem_request<4>()));
    CUDA_CHECK(cudaFuncSetAttribute(tc_stored_kernel<1, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, tcs_smem_request<4>()));
    CUDA_CHECK(cudaFuncSetAttribute(tc_stored_kernel<0, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, tcs_smem_request<8>()));
    CUDA_CHECK(cudaFuncSetAttribute(tc_stored_kernel<1, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, tcs_smem_request<8>()));
    CUDA_CHECK(cudaFuncSetAttribute(tc_sym_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTsySmemRequest));
    CUDA_CHECK(cudaFuncSetAttribute(tc_sym_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTsySmemRequest));
    CUDA_CHECK(cudaFuncSetAttribute(tc_stored_ring_kernel<0, 5, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, tcr_smem_request<5, 3>()));
    CUDA_CHECK(cudaFuncSetAttribute(tc_stored_ring_kernel<1, 5, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, tcr_smem_request<5, 3>()));
    CUDA_CHECK(cudaFuncSetAttribute(tc_cnear_kernel<kNSC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTccSmemRequest));
    done = true;
}

template <class Real, bool CPLX>
int run_tc(DevicePlan* dp, DeviceBuffers* b, int nrhs, cudaStream_t st, int& tc_launches) {
    int launches = 0;
    if (dp->n_mix > 0) {
        using S = typename Scal<Real, CPLX>::T;
        auto a = near_args<Real, CPLX>(dp, b, dp->mix_items, dp->n_mix, nrhs);
        launches += launch_near<Real, CPLX>(dp->kind, a, nrhs, ceil_div(dp->n_mix, kNearWarps), st);
        CUDA_CHECK(cudaGetLastError());
        reduce<S>(dp->tc_part_ptr, dp->tc_part_idx, (const S*)b->partial, (S*)b->U, nrhs, dp->n_tot, st);
        CUDA_CHECK(cudaGetLastError());
        ++launches;
    }
    TcArgs t;
    t.items = dp->tc_items;
    t.tiles = dp->tc_tiles;
    t.X = (const float4*)b->X;
    t.Xlo = (const float4*)b->Xlo;
    t.B = dp->tc_b;
    t.U = (float*)b->U;
    t.A = dp->tc_a;
    t.abase = dp->tc_abase;
    t.qmask = dp->tc_qmask;
    t.refs = (const BlockRef*)dp->tc_refs;
    t.isym = (const ItemSym*)dp->tc_isym;
    t.nrhs = nrhs;
    t.status = dp->status;
    t.wait_ns = dp->test_withhold ? dp->test_wait_ns : kWaitLimitNs;
    t.kappa = (float)dp->kappa;
    const int kidx = dp->kind == 0 ? 0 : 1;
    const bool stored = dp->tc_a != nullptr;
    set_tc_attributes();
    tc_launches = 0;
    if constexpr (CPLX) {
        // 3D Helmholtz: 16 complex right-hand sides per pass
        for (int r0 = 0; r0 < nrhs; r0 += kTcNc, ++launches, ++tc_launches) {
            t.r0 = r0;
            t.withhold_item = (dp->test_withhold && r0 == 0) ? 0 : -1;
            tc_bprep_kernel<true><<<(unsigned)dp->n_chunks, 256, 0, st>>>(dp->chunk_start, dp->chunk_cnt,
                                                                          (const float*)b->Q, nrhs, r0,
                                                                          (const float4*)b->X, (const float4*)b->Xlo,
                                                                          (const float4*)dp->chunk_center, dp->tc_b);
            CUDA_CHECK(cudaGetLastError());
            ++launches;
            if (r0 == 0) mark(dp, kMainEvent, st);
            tc_cnear_kernel<kNSC><<<(unsigned)dp->n_tc, kThreadsC, kTccSmemRequest, st>>>(t);
            CUDA_CHECK(cudaGetLastError());
        }
    } else {
        for (int r0 = 0; r0 < nrhs; r0 += kTcN, ++launches, ++tc_launches) {
            t.r0 = r0;
            t.withhold_item = (dp->test_withhold && r0 == 0) ? 0 : -1;
            // the pass's B operand blocks, then the translations
            tc_bprep_kernel<false><<<(unsigned)dp->n_chunks, 256, 0, st>>>(dp->chunk_start, dp->chunk_cnt, (const float*)b->Q,
                                                                   nrhs, r0, (const float4*)b->X,
                                                                   (const float4*)b->Xlo,
                                                                   (const float4*)dp->chunk_center, dp->tc_b);
            CUDA_CHECK(cudaGetLastError());
            ++launches;
            if (r0 == 0) mark(dp, kMainEvent, st);
            if (stored && dp->store_mode == 2) {
                if (kidx == 0) tc_sym_kernel<0><<<(unsigned)dp->n_tc, kTcThreads, kTsySmemRequest, st>>>(t);
                else tc_sym_kernel<1><<<(unsigned)dp->n_tc, kTcThreads, kTsySmemRequest, st>>>(t);
            } else if (stored) {
                // stages per CTA: the autotuner's choice (same arithmetic)
                const unsigned g = (unsigned)dp->n_tc;
                if (dp->tcs_stages == 5) {
                    kidx == 0 ? tc_stored_ring_kernel<0, 5, 3><<<g, kTcThreads, tcr_smem_request<5, 3>(), st>>>(t)
                              : tc_stored_ring_kernel<1, 5, 3><<<g, kTcThreads, tcr_smem_request<5, 3>(), st>>>(t);
                } else if (dp->tcs_stages == 8) {
                    kidx == 0 ? tc_stored_kernel<0, 8><<<g, kTcThreads, tcs_smem_request<8>(), st>>>(t)
                              : tc_stored_kernel<1, 8><<<g, kTcThreads, tcs_smem_request<8>(), st>>>(t);
                } else {
                    kidx == 0 ? tc_stored_kernel<0, 4><<<g, kTcThreads, tcs_smem_request<4>(), st>>>(t)
                              : tc_stored_kernel<1, 4><<<g, kTcThreads, tcs_smem_request<4>(), st>>>(t);
                }
            } else {
                // pipeline depth: the autotuner's choice (same arithmetic for every depth)
                const unsigned g = (unsigned)dp->n_tc;
                switch (dp->tc_stages) {
                    case 4: kidx == 0 ? tc_near_kernel<0, kRecNone, 4><<<g, kTcThreads, kTcSmemRequest, st>>>(t)
                                      : tc_near_kernel<1, kRecNone, 4><<<g, kTcThreads, kTcSmemRequest, st>>>(t); break;
                    case 8: kidx == 0 ? tc_near_kernel<0, kRecNone, 8><<<g, kTcThreads, kTcSmemRequest, st>>>(t)
                                      : tc_near_kernel<1, kRecNone, 8><<<g, kTcThreads, kTcSmemRequest, st>>>(t); break;
                    default: kidx == 0 ? tc_near_kernel<0, kRecNone, 6><<<g, kTcThreads, kTcSmemRequest, st>>>(t)
                                       : tc_near_kernel<1, kRecNone, 6><<<g, kTcThreads, kTcSmemRequest, st>>>(t); break;
                }
            }
            CUDA_CHECK(cudaGetLastError());
        }
    }
    dp->test_withhold = false;
    return launches;
}

template <class Real, bool CPLX>
void run_apply(DevicePlan* dp, DeviceBuffers* b, const void* q, void* u, int nrhs, bool transpose, bool use_tc,
               cudaStream_t st) {
    int launches = 0;
    using S = typename Scal<Real, CPLX>::T;
    S* Q = (S*)b->Q;
    S* U = (S*)b->U;
    const S* T = (const S*)b->T;
    const S* Tt = (const S*)b->Tt;
    S* part = (S*)b->partial;
    Range whole(transpose ? "skel apply transpose" : "skel apply");
    // 1. permute in
    mark(dp, 0, st);
    {
        Range r("permute in");
        ++launches;
        permute<S>(false, dp, (const S*)q, Q, nrhs, st);
        CUDA_CHECK(cudaGetLastError());
    }
    // 2. upward pass, levels L .. 2 (FP32_TC of a real kernel with
    // skel_options.updown_tc: the skeleton GEMMs on the tensor cores; T is
    // real, so the transposed apply is the same pass)
    const bool tc_ud = use_tc && !CPLX && sizeof(Real) == 4 && dp->ud_a_up != nullptr;
    mark(dp, 1, st);
    {
        Range r("upward pass");
        for (int l = dp->L; l >= 2; --l) {
            if (dp->up_level_ptr[l + 1] > dp->up_level_ptr[l]) {
                if (tc_ud) {
                    launches += up_down_tc(false, dp, l, reinterpret_cast<float*>(Q), nrhs, st);
                } else {
                    ++launches;
                    up_down<S>(false, dp, l, T, Q, nrhs, transpose, st);
                }
                CUDA_CHECK(cudaGetLastError());
            }
        }
    }
    // 3. near field
    mark(dp, 2, st);
    int main_launches = 0;
    {
        Range r("translations");
        const bool tc = use_tc && (!CPLX || dp->kind == 2) && sizeof(Real) == 4 && dp->n_tc > 0;
        if (tc) {
            launches += run_tc<Real, CPLX>(dp, b, nrhs, st, main_launches);
            mark(dp, 3, st);
        } else if (dp->n_items > 0) {
            auto a = near_args<Real, CPLX>(dp, b, dp->items, dp->n_items, nrhs);
            const unsigned grid = ceil_div(dp->n_items, kNearWarps);
            mark(dp, kMainEvent, st);
            main_launches = launch_near<Real, CPLX>(dp->kind, a, nrhs, grid, st);
            launches += main_launches;
            CUDA_CHECK(cudaGetLastError());
            mark(dp, 3, st);
            ++launches;
            reduce<S>(dp->part_ptr, dp->part_idx, part, U, nrhs, dp->n_tot, st);
            CUDA_CHECK(cudaGetLastError());
        } else {
            mark(dp, kMainEvent, st);
            mark(dp, 3, st);
        }
    }
    // 4. downward pass, levels 2 .. L
    mark(dp, 4, st);
    {
        Range r("downward pass");
        for (int l = 2; l <= dp->L; ++l) {
            if (dp->up_level_ptr[l + 1] > dp->up_level_ptr[l]) {
                if (tc_ud) {
                    launches += up_down_tc(true, dp, l, reinterpret_cast<float*>(U), nrhs, st);
                } else {
                    ++launches;
                    up_down<S>(true, dp, l, Tt, U, nrhs, !transpose, st);
                }
                CUDA_CHECK(cudaGetLastError());
            }
        }
    }
    // 5. permute out
    mark(dp, 5, st);
    {
        Range r("permute out");
        ++launches;
        permute<S>(true, dp, U, (S*)u, nrhs, st);
        CUDA_CHECK(cudaGetLastError());
    }
    mark(dp, 6, st);
    if (dp->prof_count < dp->prof_cap) {
        dp->prof_launches[dp->prof_count] = launches;
        dp->prof_main_launches[dp->prof_count++] = main_launches;
    }
}

// Free the stored kernel values (the plan falls back to the on-the-fly kernel).
void drop_tiles(DevicePlan* dp) {
    if (!dp->tc_a) return;
    cudaFree(dp->tc_a);
    cudaFree(dp->tc_abase);
    cudaFree(dp->tc_qmask);
    cudaFree(dp->tc_refs);
    cudaFree(dp->tc_isym);
    dp->tc_a = nullptr;
    dp->tc_abase = nullptr;
    dp->tc_qmask = nullptr;
    dp->tc_refs = nullptr;
    dp->tc_isym = nullptr;
    dp->bytes -= dp->stored_bytes + (dp->store_mode == 2 ? (int64_t)(dp->tc_refs_host.size() + dp->tc_isym_host.size())
                                                          : (int64_t)(dp->tc_abase_host.size() * sizeof(int64_t) +
                                                                      dp->tc_qmask_host.size()));
    dp->stored_bytes = 0;
    dp->store_mode = 0;
}

// Stored-operator mode `mode` (1: per-tile store, 2: symmetric store):
// evaluate the values once (the on-the-fly kernel in its fill mode, which
// also runs the translations on zero charges) into a new allocation;
// synchronous. On any failure the store is freed again.
void fill_tiles(DevicePlan* dp, cudaStream_t st, int mode) {
    if (dp->tc_a) return;
    int64_t bytes = 0;
    const int64_t floats = mode == 2 ? dp->sym_floats : dp->tile_floats;
    try {
        if (mode == 2) {
            dp->tc_refs = upload(dp->tc_refs_host, bytes);
            dp->tc_isym = upload(dp->tc_isym_host, bytes);
        } else {
            dp->tc_abase = upload(dp->tc_abase_host, bytes);
            dp->tc_qmask = upload(dp->tc_qmask_host, bytes);
        }
        dp->tc_a = dalloc<float>((size_t)floats, bytes);
    } catch (...) {
        cudaFree(dp->tc_abase);
        cudaFree(dp->tc_qmask);
        cudaFree(dp->tc_refs);
        cudaFree(dp->tc_isym);
        dp->tc_abase = nullptr;
        dp->tc_qmask = nullptr;
        dp->tc_refs = dp->tc_isym = nullptr;
        throw;
    }
    dp->store_mode = mode;
    dp->bytes += bytes;
    dp->stored_bytes = floats * (int64_t)sizeof(float);
    try {
        DeviceBuffers* b = dp->p32;
        CUDA_CHECK(cudaMemsetAsync(b->Q, 0, (size_t)dp->n_tot * sizeof(float), st));
        set_tc_attributes();
        tc_bprep_kernel<false><<<(unsigned)dp->n_chunks, 256, 0, st>>>(dp->chunk_start, dp->chunk_cnt, (const float*)b->Q, 1, 0,
                                                               (const float4*)b->X, (const float4*)b->Xlo,
                                                               (const float4*)dp->chunk_center, dp->tc_b);
        CUDA_CHECK(cudaGetLastError());
        TcArgs t;
        t.items = dp->tc_items;
        t.tiles = dp->tc_tiles;
        t.X = (const float4*)b->X;
        t.Xlo = (const float4*)b->Xlo;
        t.B = dp->tc_b;
        t.U = (float*)b->U;
        t.A = dp->tc_a;
        t.abase = dp->tc_abase;
        t.qmask = dp->tc_qmask;
        t.refs = (const BlockRef*)dp->tc_refs;
        t.isym = (const ItemSym*)dp->tc_isym;
        t.nrhs = 1;
        t.r0 = 0;
        t.status = dp->status;
        t.wait_ns = kWaitLimitNs;
        t.withhold_item = -1;
        const unsigned g = (unsigned)dp->n_tc;
        if (mode == 2) {
            if (dp->kind == 0) tc_near_kernel<0, kRecSym><<<g, kTcThreads, kTcSmemRequest, st>>>(t);
            else tc_near_kernel<1, kRecSym><<<g, kTcThreads, kTcSmemRequest, st>>>(t);
        } else {
            if (dp->kind == 0) tc_near_kernel<0, kRecTiles><<<g, kTcThreads, kTcSmemRequest, st>>>(t);
            else tc_near_kernel<1, kRecTiles><<<g, kTcThreads, kTcSmemRequest, st>>>(t);
        }
        CUDA_CHECK(cudaGetLastError());
        CUDA_CHECK(cudaStreamSynchronize(st));
        int stv = 0;
        CUDA_CHECK(cudaMemcpy(&stv, dp->status, sizeof(int), cudaMemcpyDeviceToHost));
        if (stv != 0) throw Error(-4, "the fill pass of the stored tiles timed out");
    } catch (...) {
        drop_tiles(dp);
        throw;
    }
}


// The symmetric store of the stored-operator mode (tc_kernels.cuh): the row
// chunks of every tensor-core item, and per (tile, row chunk) the stored
// block it reads. A block G(a, c) that one tile reads as (rows a, sources c)
// and another as (rows c, sources a), both with the same touching-leaf flag,
// is stored once, as (min, max), written by the first of its direct readers
// in the fill pass and read transposed by the others; every other block is
// stored for its own reader(s). Fills dp->tc_isym_host, dp->tc_refs_host,
// dp->sym_floats and dp->pairs_stored.
void plan_symmetric_store(const Layout& lay, DevicePlan* dp) {
    const int64_t nch = (int64_t)lay.chunk_start.size();
    const int64_t nitems = (int64_t)lay.tc_items.size();
    std::vector<int32_t> chunk_of(lay.n_tot, -1);
    for (int64_t c = 0; c < nch; ++c)
        for (int32_t j = 0; j < lay.chunk_cnt[c]; ++j) chunk_of[lay.chunk_start[c] + j] = (int32_t)c;
    std::vector<ItemSym> isym(nitems);
    std::vector<int32_t> rc_chunk((size_t)nitems * kMaxRc, -1);
    int64_t nref = 0;
    for (int64_t i = 0; i < nitems; ++i) {
        const TcItem& it = lay.tc_items[i];
        ItemSym& is = isym[i];
        std::memset(&is, 0, sizeof(is));
        int r = 0, m = 0;
        while (r < it.nrows) {
            const int32_t c = chunk_of[it.row_off + r];
            if (c < 0 || lay.chunk_start[c] != it.row_off + r || r + lay.chunk_cnt[c] > it.nrows || m == kMaxRc)
                throw Error(-5, "symmetric store: an item's rows are not whole chunks");
            is.ro[m] = (int16_t)r;
            rc_chunk[(size_t)i * kMaxRc + m] = c;
            r += lay.chunk_cnt[c];
            ++m;
        }
        is.ro[m] = (int16_t)it.nrows;
        is.m = m;
        is.ref0 = nref;
        nref += (int64_t)(it.list_hi - it.list_lo) * m;
    }
    if (nref >= ((int64_t)1 << 32)) throw Error(-1, "symmetric store: too many block references");
    // one request per (tile, row chunk) whose rows keep any source of the tile
    struct Req {
        uint64_t key;       // (min chunk, max chunk)
        uint32_t ref;       // its BlockRef
        uint16_t kept;      // kept (row, source) pairs of its rows
        uint8_t flags;      // 1: direct (rows = the min chunk), 2: touching leaves
        uint8_t pad;
    };
    std::vector<Req> reqs;
    reqs.reserve((size_t)nref);
    std::vector<int32_t> ref_rows(nref, 0), ref_cols(nref, 0);   // chunks of a reference: rows, sources
    for (int64_t i = 0; i < nitems; ++i) {
        const TcItem& it = lay.tc_items[i];
        const ItemSym& is = isym[i];
        for (int32_t t = it.list_lo; t < it.list_hi; ++t) {
            const SrcTile& tl = lay.tc_tiles[t];
            const int32_t c = tl.chunk;
            const uint32_t colbits = tl.cnt >= 32 ? 0xFFFFFFFFu : (1u << tl.cnt) - 1u;
            for (int k = 0; k < is.m; ++k) {
                const int32_t a = rc_chunk[(size_t)i * kMaxRc + k];
                const int lo = is.ro[k], hi = is.ro[k + 1];
                uint32_t need = 0;
                int kept = 0;
                for (int sl = 0; sl < it.nslot; ++sl) {
                    const int r0 = std::max(lo, it.slot_start[sl]), r1 = std::min(hi, it.slot_start[sl + 1]);
                    if (r1 <= r0) continue;
                    const uint32_t kb = tl.keep[sl] & colbits;
                    need |= kb;
                    kept += (r1 - r0) * __builtin_popcount(kb);
                }
                const int64_t ref = is.ref0 + (int64_t)(t - it.list_lo) * is.m + k;
                ref_rows[ref] = a;
                ref_cols[ref] = c;
                if (!need) continue;
                const uint64_t lo_c = (uint64_t)std::min(a, c), hi_c = (uint64_t)std::max(a, c);
                reqs.push_back(Req{(lo_c << 32) | hi_c, (uint32_t)ref, (uint16_t)kept,
                                   (uint8_t)((a <= c ? 1 : 0) | ((tl.flags & TASK_ADJ) ? 2 : 0)), 0});
            }
        }
    }
    std::sort(reqs.begin(), reqs.end(), [](const Req& x, const Req& y) {
        if (x.key != y.key) return x.key < y.key;
        if ((x.flags & 2) != (y.flags & 2)) return (x.flags & 2) < (y.flags & 2);
        if ((x.flags & 1) != (y.flags & 1)) return (x.flags & 1) > (y.flags & 1);   // direct readers first
        return x.ref < y.ref;
    });
    std::vector<BlockRef> refs(nref, BlockRef{0, 0u, 0, 0, 0});
    int64_t nf = 0, stored_pairs = 0;
    auto new_block = [&](int32_t rows_chunk, int32_t cols_chunk, int64_t& off, int& P) {
        P = lay.chunk_cnt[rows_chunk] | 1;
        const int64_t f = ((int64_t)P * lay.chunk_cnt[cols_chunk] + 3) & ~(int64_t)3;
        off = nf;
        nf += f;
        return f;
    };
    for (size_t g0 = 0; g0 < reqs.size();) {
        // one (pair, touching flag) group: direct readers first, then the
        // readers of the other orientation
        size_t g1 = g0;
        while (g1 < reqs.size() && reqs[g1].key == reqs[g0].key && (reqs[g1].flags & 2) == (reqs[g0].flags & 2)) ++g1;
        size_t d1 = g0;
        while (d1 < g1 && (reqs[d1].flags & 1)) ++d1;
        const Req& first = reqs[g0];
        int64_t off;
        int P;
        const int64_t f = new_block(ref_rows[first.ref], ref_cols[first.ref], off, P);
        // the first reader records the block (it reads it directly)
        for (size_t q = g0; q < g1; ++q) {
            const Req& rq = reqs[q];
            const bool same = ref_rows[rq.ref] == ref_rows[first.ref];    // same orientation as stored
            refs[rq.ref] = BlockRef{off, (uint32_t)(4 * f), (uint16_t)P,
                                    (uint8_t)((same ? 0 : kRefTransposed) | (q == g0 ? kRefRecord : 0)), 0};
            if (same) stored_pairs += rq.kept;
        }
        (void)d1;
        g0 = g1;
    }
    // every block fits the place of its reader's row chunk in a stage (rows
    // ro_k .. ro_{k+1} at float (ro_k + k) * 32, up to the next chunk's place)
    for (int64_t i = 0; i < nitems; ++i) {
        const TcItem& it = lay.tc_items[i];
        const ItemSym& is = isym[i];
        for (int32_t t = it.list_lo; t < it.list_hi; ++t)
            for (int k = 0; k < is.m; ++k) {
                const BlockRef& rf = refs[is.ref0 + (int64_t)(t - it.list_lo) * is.m + k];
                if (rf.bytes == 0) continue;
                const int64_t cap = 4 * 32 * (int64_t)(is.ro[k + 1] - is.ro[k] + 1);
                if ((int64_t)rf.bytes > cap || rf.bytes % 16 != 0 || rf.off % 4 != 0 || rf.off + rf.bytes / 4 > nf)
                    throw Error(-5, "symmetric store: a block does not fit its row chunk's place");
            }
    }
    dp->tc_isym_host.resize(isym.size() * sizeof(ItemSym));
    std::memcpy(dp->tc_isym_host.data(), isym.data(), dp->tc_isym_host.size());
    dp->tc_refs_host.resize(refs.size() * sizeof(BlockRef));
    std::memcpy(dp->tc_refs_host.data(), refs.data(), dp->tc_refs_host.size());
    dp->sym_floats = nf;
    dp->pairs_stored = stored_pairs;
}

}  // namespace

// The tensor-core up/down work items of one direction and their A blobs (see
// tc_updown.cuh): per level, per box, per 128 output rows; upward A(i, j) =
// T(i, j), downward A(j, i) = T(i, j) (real T, column-major k x (n - k)).
// A downward box without redundant rows still gets one item (no rows, no
// tiles) for its u_S += uhat.
void build_ud_items(bool down, const std::vector<UpBox>& up, const std::vector<int64_t>& level_ptr, const Layout& lay,
                    std::vector<UdItem>& items, std::vector<int64_t>& ptr, std::vector<float>& A) {
    ptr.assign(level_ptr.size(), 0);
    for (size_t l = 0; l + 1 < level_ptr.size(); ++l) {
        ptr[l] = (int64_t)items.size();
        for (int64_t b = level_ptr[l]; b < level_ptr[l + 1]; ++b) {
            const UpBox& u = up[b];
            const int k = u.k, r = u.n - u.k;
            const int nout = down ? r : k, ninner = down ? k : r;
            const int ntile = (ninner + 31) / 32;
            if (nout == 0) {
                if (down) items.push_back(UdItem{(int64_t)A.size(), (int32_t)b, 0, 0, 0});
                continue;
            }
            for (int row0 = 0; row0 < nout; row0 += 128) {
                const int nrows = std::min(128, nout - row0);
                items.push_back(UdItem{(int64_t)A.size(), (int32_t)b, row0, nrows, ntile});
                for (int t = 0; t < ntile; ++t) {
                    const size_t base = A.size();
                    A.resize(base + (size_t)ud_blob_floats(nrows), 0.f);
                    for (int jj = 0; jj < 32; ++jj) {
                        const int j = 32 * t + jj;                     // inner index
                        int32_t e = -1;
                        if (j < ninner) {
                            e = (int32_t)(down ? u.dst + j : u.off + lay.pos[u.off + k + j]);
                            for (int row = 0; row < nrows; ++row) {
                                const int o = row0 + row;              // output index
                                const double v = down ? lay.T[u.T_off + j + (int64_t)o * k]
                                                      : lay.T[u.T_off + o + (int64_t)j * k];
                                A[base + ((size_t)(jj / 4) * nrows + row) * 4 + jj % 4] = (float)v;
                            }
                        }
                        std::memcpy(&A[base + (size_t)nrows * 32 + jj], &e, sizeof(e));
                    }
                }
            }
        }
    }
    ptr.back() = (int64_t)items.size();
}

DevicePlan* device_plan_create(const Plan& p, const Layout& lay, int nrhs_max, int store_tiles, int store_stages,
                               bool updown_tc) {
    DevicePlan* dp = new DevicePlan();
    dp->tcs_stages = store_stages == 8 || store_stages == 5 ? store_stages : 4;
    try {
        CUDA_CHECK(cudaGetDevice(&dp->device));
        dp->dim = p.tree.dim;
        dp->kind = p.kind;
        dp->kappa = p.kappa;
        dp->cplx = p.kind == 2 || p.kind == 3;
        dp->N = p.tree.n;
        dp->n_tot = lay.n_tot;
        dp->nrhs_max = nrhs_max;
        dp->top = lay.top;
        dp->L = p.tree.L;
        dp->box_off = upload(lay.box_off, dp->bytes);
        dp->box_n = upload(lay.box_n, dp->bytes);
        dp->box_nslot = upload(lay.box_nslot, dp->bytes);
        dp->slot_start = upload(lay.slot_start, dp->bytes);
        dp->pos = upload(lay.pos, dp->bytes);
        {
            std::vector<int64_t> eop(dp->N, -1);
            for (size_t i = 0; i < lay.perm_point.size(); ++i) eop[lay.perm_point[i]] = lay.perm_entry[i];
            for (int64_t v : eop)
                if (v < 0) throw Error(-5, "a point has no leaf entry");
            dp->eop = upload(eop, dp->bytes);
        }
        // leaf boxes with no redundant index (k = |I_B|): their upward and
        // downward steps move to the permutations (eop2, see permute_in);
        // the level launches get the other boxes
        std::vector<UpBox> up;
        dp->up_level_ptr.assign(lay.up_level_ptr.size(), 0);
        {
            std::vector<int64_t> point_of(lay.n_tot, -1), eop2(dp->N, -1);
            for (size_t i = 0; i < lay.perm_entry.size(); ++i) point_of[lay.perm_entry[i]] = lay.perm_point[i];
            int64_t fused = 0;
            for (size_t l = 0; l + 1 < lay.up_level_ptr.size(); ++l) {
                dp->up_level_ptr[l] = (int64_t)up.size();
                for (int64_t i = lay.up_level_ptr[l]; i < lay.up_level_ptr[l + 1]; ++i) {
                    const UpBox& u = lay.up[i];
                    bool fuse = u.k == u.n && i < (int64_t)lay.up_leaf.size() && lay.up_leaf[i];
                    for (int j = 0; fuse && j < u.k; ++j) {
                        const int64_t p = point_of[u.off + lay.pos[u.off + j]];
                        fuse = p >= 0 && eop2[p] < 0;
                    }
                    if (!fuse) {
                        up.push_back(u);
                        continue;
                    }
                    for (int j = 0; j < u.k; ++j) eop2[point_of[u.off + lay.pos[u.off + j]]] = u.dst + j;
                    ++fused;
                }
            }
            dp->up_level_ptr.back() = (int64_t)up.size();
            if (fused > 0) dp->eop2 = upload(eop2, dp->bytes);
        }
        dp->up = upload(up, dp->bytes);
        if (!dp->cplx) {
            // padded FP32 copies of T for the vectorised up/down copies
            std::vector<float> tp, ttp;
            std::vector<int64_t> tpo(up.size()), ttpo(up.size());
            for (size_t b = 0; b < up.size(); ++b) {
                const UpBox& ub = up[b];
                const int k = ub.k, r = ub.n - ub.k, ldk = (k + 3) & ~3, ldr = (r + 3) & ~3;
                tpo[b] = (int64_t)tp.size();
                tp.resize(tp.size() + (size_t)ldk * r, 0.f);
                for (int j = 0; j < r; ++j)
                    for (int i = 0; i < k; ++i) tp[tpo[b] + i + (size_t)j * ldk] = (float)lay.T[ub.T_off + i + (int64_t)j * k];
                ttpo[b] = (int64_t)ttp.size();
                ttp.resize(ttp.size() + (size_t)ldr * k, 0.f);
                for (int i = 0; i < k; ++i)
                    for (int j = 0; j < r; ++j) ttp[ttpo[b] + j + (size_t)i * ldr] = (float)lay.T[ub.T_off + i + (int64_t)j * k];
            }
            // work lists of the CTA-wide kernel, per direction and rows per CTA
            for (int dir = 0; dir < 2; ++dir)
                for (int wi = 0; wi < 4; ++wi) {
                    const int rows = 32 << wi;
                    std::vector<int2> w;
                    std::vector<int64_t>& wp = dp->ud_work_ptr[dir][wi];
                    wp.assign(dp->up_level_ptr.size(), 0);
                    for (size_t l = 0; l + 1 < dp->up_level_ptr.size(); ++l) {
                        wp[l] = (int64_t)w.size();
                        for (int64_t b = dp->up_level_ptr[l]; b < dp->up_level_ptr[l + 1]; ++b) {
                            const int nout = dir ? up[b].n - up[b].k : up[b].k;
                            const int nblk = std::max(dir ? 1 : 0, (nout + rows - 1) / rows);
                            for (int i = 0; i < nblk; ++i) w.push_back(make_int2((int)b, i * rows));
                        }
                    }
                    wp.back() = (int64_t)w.size();
                    dp->ud_work[dir][wi] = upload(w, dp->bytes);
                }
            dp->ud_tp = upload(tp, dp->bytes);
            dp->ud_ttp = upload(ttp, dp->bytes);
            dp->ud_tp_off = upload(tpo, dp->bytes);
            dp->ud_ttp_off = upload(ttpo, dp->bytes);
        }
        if (!dp->cplx && updown_tc) {
            for (int down = 0; down < 2; ++down) {
                std::vector<UdItem> items;
                std::vector<float> A;
                build_ud_items(down != 0, up, dp->up_level_ptr, lay, items, down ? dp->ud_ptr_down : dp->ud_ptr_up, A);
                (down ? dp->ud_items_down : dp->ud_items_up) = upload(items, dp->bytes);
                (down ? dp->ud_a_down : dp->ud_a_up) = upload(A, dp->bytes);
            }
        }
        const int nl = (int)dp->up_level_ptr.size() - 1;
        dp->up_level_maxk.assign(std::max(nl, 0), 0);
        dp->up_level_maxr.assign(std::max(nl, 0), 0);
        for (int l = 0; l < nl; ++l)
            for (int64_t i = dp->up_level_ptr[l]; i < dp->up_level_ptr[l + 1]; ++i) {
                dp->up_level_maxk[l] = std::max(dp->up_level_maxk[l], up[i].k);
                dp->up_level_maxr[l] = std::max(dp->up_level_maxr[l], up[i].n - up[i].k);
            }
        dp->task_src = upload(lay.task_src, dp->bytes);
        dp->task_mask = upload(lay.task_mask, dp->bytes);
        dp->task_flags = upload(lay.task_flags, dp->bytes);
        dp->items = upload(lay.items, dp->bytes);
        dp->n_items = (int64_t)lay.items.size();
        dp->part_ptr = upload(lay.part_ptr, dp->bytes);
        dp->part_idx = upload(lay.part_idx, dp->bytes);
        dp->mix_items = upload(lay.mix_items, dp->bytes);
        dp->n_mix = (int64_t)lay.mix_items.size();
        dp->tc_tiles = upload(lay.tc_tiles, dp->bytes);
        dp->tc_items = upload(lay.tc_items, dp->bytes);
        dp->n_tc = (int64_t)lay.tc_items.size();
        if (dp->n_tc > 0 && (!dp->cplx || dp->kind == 2)) {
            dp->chunk_start = upload(lay.chunk_start, dp->bytes);
            dp->chunk_cnt = upload(lay.chunk_cnt, dp->bytes);
            dp->chunk_center = upload(lay.chunk_center, dp->bytes);
            dp->n_chunks = (int64_t)lay.chunk_start.size();
            dp->tc_b = dalloc<float>((size_t)dp->n_chunks * (dp->cplx ? kChunkFloatsC : kChunkFloats), dp->bytes);
        }
        dp->tc_n_slots = lay.tc_n_slots;
        dp->tc_part_ptr = upload(lay.tc_part_ptr, dp->bytes);
        dp->tc_part_idx = upload(lay.tc_part_idx, dp->bytes);
        dp->status = dalloc<int>(1, dp->bytes);
        CUDA_CHECK(cudaMemset(dp->status, 0, sizeof(int)));
        dp->p64 = new DeviceBuffers();
        make_buffers<double>(dp, lay, dp->p64);
        dp->p32 = new DeviceBuffers();
        make_buffers<float>(dp, lay, dp->p32);
        if (dp->n_tc > 0 && !dp->cplx) {
            dp->n_tc_tiles = (int64_t)lay.tc_tiles.size();
            for (const TcItem& it : lay.tc_items)
                if (it.nrows < 1 || it.nrows > kTcRows) throw Error(-5, "tensor-core item with no rows");
            // per-tile store: each item's tiles back to back; a tile keeps the
            // 4-column quads in which some row of its item keeps a source
            // (the others are zero in every row), nrows float4 each
            dp->tc_abase_host.resize(lay.tc_items.size());
            dp->tc_qmask_host.assign(lay.tc_tiles.size(), 0);
            int64_t nf = 0;
            for (size_t i = 0; i < lay.tc_items.size(); ++i) {
                const TcItem& it = lay.tc_items[i];
                dp->tc_abase_host[i] = nf;
                for (int32_t t = it.list_lo; t < it.list_hi; ++t) {
                    uint32_t cm = 0;
                    for (int sl = 0; sl < it.nslot; ++sl)
                        if (std::min(it.slot_start[sl + 1], it.nrows) > std::max(it.slot_start[sl], 0))
                            cm |= lay.tc_tiles[t].keep[sl];
                    uint32_t qm = 0;
                    for (int q = 0; q < 8; ++q)
                        if ((cm >> (4 * q)) & 0xFu) qm |= 1u << q;
                    dp->tc_qmask_host[t] = (uint8_t)qm;
                    nf += (int64_t)__builtin_popcount(qm) * it.nrows * 4;
                }
            }
            dp->tile_floats = nf;
            plan_symmetric_store(lay, dp);
            if (store_tiles) fill_tiles(dp, 0, store_tiles == 2 ? 2 : 1);
        }
        CUDA_CHECK(cudaDeviceSynchronize());
    } catch (...) {
        device_plan_destroy(dp);
        throw;
    }
    return dp;
}

void device_plan_destroy(DevicePlan* dp) {
    if (!dp) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(dp->device);
    void* ptrs[] = {dp->box_off, dp->box_n, dp->box_nslot, dp->slot_start, dp->pos, dp->eop, dp->eop2, dp->up, dp->task_src, dp->task_mask, dp->task_flags, dp->items,
                    dp->part_ptr, dp->part_idx, dp->stage_in, dp->stage_out, dp->mix_items, dp->tc_tiles,
                    dp->tc_items, dp->tc_part_ptr, dp->tc_part_idx, dp->status,
                    dp->chunk_start, dp->chunk_cnt, dp->chunk_center, dp->tc_b, dp->tc_a, dp->tc_abase,
                    dp->tc_qmask, dp->tc_refs, dp->tc_isym, dp->ud_items_up, dp->ud_items_down,
                    dp->ud_a_up, dp->ud_a_down, dp->ud_tp, dp->ud_ttp, dp->ud_tp_off, dp->ud_ttp_off};
    for (void* p : ptrs) cudaFree(p);
    for (int dir = 0; dir < 2; ++dir)
        for (int wi = 0; wi < 4; ++wi) cudaFree(dp->ud_work[dir][wi]);
    for (void* e : dp->events)
        if (e) cudaEventDestroy((cudaEvent_t)e);
    free_buffers(dp->p64);
    free_buffers(dp->p32);
    cudaSetDevice(cur);
    delete dp;
}

void device_set_profiling(DevicePlan* dp, int max_applies) {
    if (max_applies < 0 || max_applies > 100000) throw Error(-1, "max_applies out of range");
    while ((int)dp->events.size() < kProfEvents * max_applies) {
        cudaEvent_t e;
        CUDA_CHECK(cudaEventCreate(&e));
        dp->events.push_back((void*)e);
    }
    dp->prof_cap = max_applies;
    dp->prof_count = 0;
    dp->prof_launches.assign(max_applies, 0);
    dp->prof_main_launches.assign(max_applies, 0);
}

int device_status(DevicePlan* dp) {
    int v = 0;
    CUDA_CHECK(cudaDeviceSynchronize());
    CUDA_CHECK(cudaMemcpy(&v, dp->status, sizeof(int), cudaMemcpyDeviceToHost));
    CUDA_CHECK(cudaMemset(dp->status, 0, sizeof(int)));
    return v;
}

void device_last_timings(DevicePlan* dp, double* ms6, int* launches, int* n_applies, double* ms_main,
                         int* main_launches) {
    if (dp->prof_cap == 0) throw Error(-6, "profiling is not enabled");
    for (int i = 0; i < 6; ++i) ms6[i] = 0;
    *launches = 0;
    *ms_main = 0;
    *main_launches = 0;
    for (int a = 0; a < dp->prof_count; ++a) {
        cudaEvent_t* ev = (cudaEvent_t*)&dp->events[a * kProfEvents];
        CUDA_CHECK(cudaEventSynchronize(ev[6]));
        for (int i = 0; i < 6; ++i) {
            float ms = 0;
            CUDA_CHECK(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
            ms6[i] += ms;
        }
        float ms = 0;
        CUDA_CHECK(cudaEventElapsedTime(&ms, ev[kMainEvent], ev[3]));
        *ms_main += ms;
        *launches += dp->prof_launches[a];
        *main_launches += dp->prof_main_launches[a];
    }
    *n_applies = dp->prof_count;
}

void device_apply(DevicePlan* dp, const void* q, void* u, int nrhs, int precision, bool transpose,
                  void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == 0) {
        if (dp->cplx) run_apply<double, true>(dp, dp->p64, q, u, nrhs, transpose, false, st);
        else run_apply<double, false>(dp, dp->p64, q, u, nrhs, transpose, false, st);
    } else if (dp->cplx) {
        // tensor-core translations for 3D Helmholtz, one pass per 16 right-hand sides
        const bool tc = precision == 2 && nrhs >= 4 && dp->kind == 2;
        run_apply<float, true>(dp, dp->p32, q, u, nrhs, transpose, tc, st);
    } else if (precision == 2 && nrhs >= 4) {
        // tensor-core translations, one pass per 32 right-hand sides
        run_apply<float, false>(dp, dp->p32, q, u, nrhs, transpose, true, st);
    } else {
        run_apply<float, false>(dp, dp->p32, q, u, nrhs, transpose, false, st);
    }
}

TuneReport device_autotune(DevicePlan* dp, int nrhs, bool allow_store, void* stream) {
    if (dp->cplx) throw Error(-1, "autotune: real kernels only");
    if (nrhs < 1 || nrhs > dp->nrhs_max) throw Error(-1, "autotune: nrhs must be in [1, nrhs_max]");
    cudaStream_t st = (cudaStream_t)stream;
    TuneReport rep;
    const int saved_cap = dp->prof_cap;
    dp->prof_cap = 0;                                      // no profiling events while measuring
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float* keep_a = nullptr;                               // stored blocks hidden while timing
    try {
        CUDA_CHECK(cudaEventCreate(&e0));
        CUDA_CHECK(cudaEventCreate(&e1));
        DeviceBuffers* b = dp->p32;
        const size_t qbytes = (size_t)dp->n_tot * dp->nrhs_max * sizeof(float);
        CUDA_CHECK(cudaMemsetAsync(b->Q, 0, qbytes, st));  // zero data: timing only, nothing grows
        CUDA_CHECK(cudaMemsetAsync(b->U, 0, qbytes, st));
        auto time_ms = [&](auto&& launch, int reps) {
            launch();                                      // warm-up
            CUDA_CHECK(cudaEventRecord(e0, st));
            for (int i = 0; i < reps; ++i) launch();
            CUDA_CHECK(cudaEventRecord(e1, st));
            CUDA_CHECK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
            CUDA_CHECK(cudaGetLastError());
            return (double)ms / reps;
        };
        // 1. up/down launch shape per level: warps per CTA (every choice
        //    adds the same partial sums in the same order)
        const int nl = (int)dp->up_level_ptr.size() - 1;
        dp->ud_warps_up.assign(std::max(nl, 0), 0);
        dp->ud_warps_down.assign(std::max(nl, 0), 0);
        for (int l = 2; l <= dp->L && l < nl; ++l) {
            if (dp->up_level_ptr[l + 1] == dp->up_level_ptr[l]) continue;
            for (int down = 0; down < 2; ++down) {
                std::vector<int8_t>& t = down ? dp->ud_warps_down : dp->ud_warps_up;
                const float* T = (const float*)(down ? b->Tt : b->T);
                const int ninner = down ? dp->up_level_maxk[l] : dp->up_level_maxr[l];
                const int def = ud_default_warps((ninner + kGT - 1) / kGT);
                double best_ms = 1e30, def_ms = 0;
                int best = def;
                for (int W : {1, 2, 4, 8, kUdAsync + 1, kUdAsync + 2, kUdAsync + 4, kUdAsync + 8}) {
                    const double ms = time_ms([&] { up_down<float>(down != 0, dp, l, T, (float*)(down ? b->U : b->Q),
                                                                   nrhs, down != 0, st, W); }, 5);
                    if (W == def) def_ms = ms;
                    if (ms < best_ms) best_ms = ms, best = W;
                }
                t[l] = (int8_t)best;
                rep.ms_updown_default += def_ms;
                rep.ms_updown_tuned += best_ms;
                rep.n_changed += best != def;
                ++rep.n_levels;
            }
        }
        // 2. tensor-core translations: on the fly or stored tiles
        if (dp->n_tc > 0 && nrhs >= 4) {
            int passes = 0;
            auto tc = [&] { run_tc<float, false>(dp, b, nrhs, st, passes); };
            keep_a = dp->tc_a;
            dp->tc_a = nullptr;                            // time the on-the-fly kernel
            // its pipeline depth (bulk-copy stages): the fastest of 4, 6, 8
            rep.ms_onfly = 1e30;
            int best_ns = kNS;
            for (int ns : {4, 6, 8}) {
                dp->tc_stages = ns;
                const double ms = time_ms(tc, 3);
                if (ms < rep.ms_onfly) rep.ms_onfly = ms, best_ns = ns;
            }
            dp->tc_stages = best_ns;
            rep.tc_stages = best_ns;
            dp->tc_a = keep_a;
            keep_a = nullptr;
            // the stores: the one the plan holds, and (allow_store) each one
            // that fits the free memory with 2 GB to spare, timed in turn; the
            // fastest of on the fly, per-tile and symmetric is kept
            double best = rep.ms_onfly;
            int best_mode = 0;
            for (int mode : {1, 2}) {
                if (!(dp->tc_a && dp->store_mode == mode)) {
                    if (!allow_store) continue;
                    drop_tiles(dp);
                    size_t free_b = 0, total_b = 0;
                    CUDA_CHECK(cudaMemGetInfo(&free_b, &total_b));
                    const int64_t floats = mode == 2 ? dp->sym_floats : dp->tile_floats;
                    if (free_b <= (size_t)floats * sizeof(float) + ((size_t)2 << 30)) continue;
                    fill_tiles(dp, st, mode);
                }
                double ms = time_ms(tc, 3);
                if (mode == 1) {
                    // the per-tile store's kernel form: 4 stages (two CTAs per
                    // SM), 8 (one), or 5 value + 3 operand slots (split rings)
                    int best_stages = dp->tcs_stages;
                    for (int ns : {4, 8, 5}) {
                        if (ns == best_stages) continue;
                        const int keep_stages = dp->tcs_stages;
                        dp->tcs_stages = ns;
                        const double ms2 = time_ms(tc, 3);
                        if (ms2 < ms) ms = ms2, best_stages = ns;
                        dp->tcs_stages = keep_stages;
                    }
                    dp->tcs_stages = best_stages;
                    rep.tcs_stages = best_stages;
                }
                (mode == 2 ? rep.ms_sym : rep.ms_stored) = ms;
                if (ms < best) best = ms, best_mode = mode;
            }
            if (dp->store_mode != best_mode) {
                drop_tiles(dp);
                if (best_mode) fill_tiles(dp, st, best_mode);
            }
            rep.stored = dp->store_mode;
        }
    } catch (...) {
        dp->prof_cap = saved_cap;
        if (keep_a) dp->tc_a = keep_a;
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        throw;
    }
    dp->prof_cap = saved_cap;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rep;
}

}  // namespace skel
