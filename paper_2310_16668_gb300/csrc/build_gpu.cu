// Algorithm 1 (strong recursive skeletonization) on the GPU, FP64 / complex128.
//
// The same steps as the host build, per level L..2 (Section 2.1):
//   I_B  from the children's skeletons (host: integer bookkeeping only);
//   M    = [G(P, I_B); conj G(P, I_B)] for the proxy points P (real kernels:
//          the first block), evaluated on the device;
//   column-pivoted Householder QR of M, stopped at the first |R_jj| <=
//          tol |R_00|, column norms recomputed from the updated columns at
//          every step (no downdating), pivot ties to the lowest index;
//   T    = R_11^{-1} R_12 by back substitution, in place over R_12.
//
// id_kernel: one CTA per box. The box's matrix lives in a global workspace
// (column-major, m rows); the CTA keeps the Householder vector, R's diagonal
// and the column norms in shared memory. Per step: a block argmax over the
// norms, the column swap, the reflector, then every trailing column gets its
// dot product, update and new norm from one warp (lanes over rows, so each
// column is read and written once, coalesced). id_gather_kernel then packs
// every box's T (k x r, column-major) at offsets the host computed from the
// ranks, so only T, the pivots and the ranks come back to the host.
//
// Work per box: sum_j (n - j - 1)(m - j) x 6 flops (real; x 4 for complex),
// a few passes over the box's m x n matrix per step; FP64 arithmetic
// throughout (the ranks are decided at tolerances down to 1e-12).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>

#include "device.h"
#include "host.h"

namespace skel {

namespace {

#define BCHECK(x)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (x);                                                            \
        if (e_ != cudaSuccess)                                                           \
            throw Error(-3, std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x); \
    } while (0)

constexpr int kIdThreads = 256;
constexpr int kIdWarps = kIdThreads / 32;

struct Zd {
    double re, im;
};
__device__ inline Zd operator+(Zd a, Zd b) { return {a.re + b.re, a.im + b.im}; }
__device__ inline Zd operator-(Zd a, Zd b) { return {a.re - b.re, a.im - b.im}; }
__device__ inline Zd operator*(Zd a, Zd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ inline Zd operator*(double s, Zd a) { return {s * a.re, s * a.im}; }
__device__ inline Zd operator/(Zd a, Zd b) {
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__device__ inline double sq(double v) { return v * v; }
__device__ inline double sq(Zd v) { return v.re * v.re + v.im * v.im; }
__device__ inline double cj(double v) { return v; }
__device__ inline Zd cj(Zd v) { return {v.re, -v.im}; }
template <class S> __device__ inline S zero_of();
template <> __device__ inline double zero_of<double>() { return 0.0; }
template <> __device__ inline Zd zero_of<Zd>() { return {0.0, 0.0}; }
__device__ inline double from_real(double v, double) { return v; }
__device__ inline Zd from_real(double v, Zd) { return {v, 0.0}; }
__device__ inline double unit_dir(double x0, double ax0) { return x0 / ax0; }
__device__ inline Zd unit_dir(Zd x0, double ax0) { return {x0.re / ax0, x0.im / ax0}; }

__device__ inline double wsum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline Zd wsum(Zd v) { return {wsum(v.re), wsum(v.im)}; }

// Green's functions of Eq. 2 (and the 2D Helmholtz kernel), zero at r = 0.
template <int KIND> struct Gd;
template <> struct Gd<0> {
    using S = double;
    __device__ static S at(double r2, double) { return r2 == 0.0 ? 0.0 : -log(sqrt(r2)) / (2.0 * M_PI); }
};
template <> struct Gd<1> {
    using S = double;
    __device__ static S at(double r2, double) { return r2 == 0.0 ? 0.0 : 1.0 / (4.0 * M_PI * sqrt(r2)); }
};
template <> struct Gd<2> {
    using S = Zd;
    __device__ static S at(double r2, double kappa) {
        if (r2 == 0.0) return {0.0, 0.0};
        const double r = sqrt(r2);
        double s, c;
        sincos(kappa * r, &s, &c);
        const double w = 1.0 / (4.0 * M_PI * r);
        return {c * w, s * w};
    }
};
template <> struct Gd<3> {
    using S = Zd;
    __device__ static S at(double r2, double kappa) {
        if (r2 == 0.0) return {0.0, 0.0};
        const double kr = kappa * sqrt(r2);
        return {-0.25 * y0(kr), 0.25 * j0(kr)};
    }
};

struct IdArgs {
    const double* pts;        // n_points x dim
    const int64_t* I;         // point indices of every box's I_B, concatenated
    const int64_t* box_ptr;   // nbox + 1
    const double* cen;        // 3 per box
    const double* prox;       // np x dim proxy offsets from the box centre
    const int64_t* ws_off;    // nbox: first workspace element of each box
    void* ws;                 // m x n per box, column-major
    int32_t* k_out;           // nbox
    int32_t* piv_out;         // per entry: local column index, S first
    int dim, np, m, n_max;
    double kappa, tol;
};

// NT threads per CTA: 256 on levels with many boxes, 1024 where few boxes
// (the top levels) would leave most SMs idle
template <int KIND, int NT>
__global__ void __launch_bounds__(NT) id_kernel(IdArgs A) {
    constexpr int kW = NT / 32;
    using S = typename Gd<KIND>::S;
    extern __shared__ __align__(16) unsigned char id_smem[];
    S* v = reinterpret_cast<S*>(id_smem);                  // m
    S* rdiag = v + A.m;                                     // m
    double* nrm = reinterpret_cast<double*>(rdiag + A.m);   // n_max
    __shared__ double red_v[kW];
    __shared__ int red_i[kW];
    __shared__ int sh_p;
    __shared__ double sh_sum;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = blockIdx.x;
    const int64_t e0 = A.box_ptr[b];
    const int n = (int)(A.box_ptr[b + 1] - e0);
    const int m = A.m, np = A.np, dim = A.dim;
    S* M = reinterpret_cast<S*>(A.ws) + A.ws_off[b];
    const int64_t* I = A.I + e0;
    int32_t* piv = A.piv_out + e0;

    // proxy matrix: rows = proxy points (then their conjugates), columns = I_B
    for (int64_t e = tid; e < (int64_t)m * n; e += NT) {
        const int j = (int)(e / m), i = (int)(e - (int64_t)j * m);
        const int ip = i < np ? i : i - np;
        const double* x = A.pts + I[j] * dim;
        double r2 = 0.0;
        for (int d = 0; d < dim; ++d) {
            const double y = A.cen[b * 3 + d] + A.prox[ip * dim + d];
            const double dd = y - x[d];
            r2 += dd * dd;
        }
        S g = Gd<KIND>::at(r2, A.kappa);
        if (i >= np) g = cj(g);
        M[e] = g;
    }
    for (int c = tid; c < n; c += NT) piv[c] = c;
    __syncthreads();
    for (int c = warp; c < n; c += kW) {
        const S* col = M + (size_t)c * m;
        double s = 0.0;
        for (int i = lane; i < m; i += 32) s += sq(col[i]);
        s = wsum(s);
        if (lane == 0) nrm[c] = s;
    }
    __syncthreads();

    const int kmax = min(m, n);
    int k = kmax;
    bool zero = false;
    double r00 = 0.0;
    for (int j = 0; j < kmax; ++j) {
        // pivot: the largest remaining norm, ties to the lowest index
        double bv = -1.0;
        int bi = n;
        for (int c = j + tid; c < n; c += NT)
            if (nrm[c] > bv) { bv = nrm[c]; bi = c; }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (lane == 0) { red_v[warp] = bv; red_i[warp] = bi; }
        __syncthreads();
        if (tid == 0) {
            double wv = red_v[0];
            int wi = red_i[0];
            for (int w = 1; w < kW; ++w)
                if (red_v[w] > wv || (red_v[w] == wv && red_i[w] < wi)) { wv = red_v[w]; wi = red_i[w]; }
            sh_p = wi;
        }
        __syncthreads();
        const int p = sh_p;
        if (p >= n || !isfinite(nrm[p])) {   // only non-finite norms leave no candidate
            if (tid == 0) A.k_out[b] = -1;
            return;
        }
        const double cn = sqrt(nrm[p]);
        if (j == 0) r00 = cn;
        if (j == 0 && cn == 0.0) { zero = true; break; }
        if (cn == 0.0 || !(cn > A.tol * r00)) { k = j; break; }
        // swap columns j and p (every row: rows above j hold R), keeping the
        // pivot column's trailing part as the reflector's vector
        for (int i = tid; i < m; i += NT) {
            const S pv = M[(size_t)p * m + i];
            if (p != j) {
                M[(size_t)p * m + i] = M[(size_t)j * m + i];
                M[(size_t)j * m + i] = pv;
            }
            if (i >= j) v[i] = pv;
        }
        __syncthreads();
        if (tid == 0 && p != j) {
            const int32_t tp = piv[j];
            piv[j] = piv[p];
            piv[p] = tp;
            const double tn = nrm[j];
            nrm[j] = nrm[p];
            nrm[p] = tn;
        }
        const S x0 = v[j];
        const double ax0 = sqrt(sq(x0));
        const S alpha = ax0 == 0.0 ? from_real(-cn, x0) : (-cn) * unit_dir(x0, ax0);
        __syncthreads();
        if (tid == 0) {
            v[j] = x0 - alpha;
            rdiag[j] = alpha;
        }
        __syncthreads();
        double part = 0.0;
        for (int i = j + tid; i < m; i += NT) part += sq(v[i]);
        part = wsum(part);
        if (lane == 0) red_v[warp] = part;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < kW; ++w) s += red_v[w];
            sh_sum = s;
        }
        __syncthreads();
        const double vn2 = sh_sum;
        if (vn2 > 0.0) {
            const double two = 2.0 / vn2;
            for (int c = j + 1 + warp; c < n; c += kW) {
                S* col = M + (size_t)c * m;
                S dot = zero_of<S>();
                for (int i = j + lane; i < m; i += 32) dot = dot + cj(v[i]) * col[i];
                dot = wsum(dot);
                const S f = two * dot;
                double s = 0.0;
                for (int i = j + lane; i < m; i += 32) {
                    const S val = col[i] - f * v[i];
                    col[i] = val;
                    if (i > j) s += sq(val);
                }
                s = wsum(s);
                if (lane == 0) nrm[c] = s;
            }
        }
        __syncthreads();
    }
    if (zero) {
        if (tid == 0) A.k_out[b] = n;
        return;
    }
    if (k < 1) k = 1;
    // T = R_11^{-1} R_12, in place over rows 0..k-1 of columns k..n-1
    for (int c = k + tid; c < n; c += NT) {
        S* col = M + (size_t)c * m;
        for (int i = k - 1; i >= 0; --i) {
            S acc = col[i];
            for (int s = i + 1; s < k; ++s) acc = acc - M[(size_t)s * m + i] * col[s];
            col[i] = acc / rdiag[i];
        }
    }
    if (tid == 0) A.k_out[b] = k;
}

template <class S>
__global__ void __launch_bounds__(kIdThreads) id_gather_kernel(const S* ws, const int64_t* ws_off,
                                                               const int64_t* box_ptr, int m,
                                                               const int32_t* k_in, const int64_t* T_off,
                                                               S* T_out) {
    const int b = blockIdx.x;
    const int n = (int)(box_ptr[b + 1] - box_ptr[b]);
    const int k = k_in[b];
    const int r = n - k;
    if (r <= 0 || k <= 0) return;
    const S* M = ws + ws_off[b];
    S* T = T_out + T_off[b];
    for (int64_t e = threadIdx.x; e < (int64_t)k * r; e += kIdThreads) {
        const int c = (int)(e / k), i = (int)(e - (int64_t)c * k);
        T[e] = M[(size_t)(k + c) * m + i];
    }
}

// device buffer that grows on demand (build time only)
struct DBuf {
    void* p = nullptr;
    size_t cap = 0;
    void* get(size_t bytes) {
        if (bytes > cap) {
            if (p) cudaFree(p);
            p = nullptr;
            cap = 0;
            if (alloc_should_fail()) throw Error(-2, "cudaMalloc failed in the device build: simulated (test hook)");
            cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
            if (e != cudaSuccess) {
                cudaGetLastError();
                throw Error(-2, std::string("cudaMalloc failed in the device build: ") + cudaGetErrorString(e));
            }
            cap = bytes;
        }
        return p;
    }
    ~DBuf() {
        if (p) cudaFree(p);
    }
};

template <class T>
T* put(DBuf& buf, const std::vector<T>& v) {
    T* p = (T*)buf.get(v.size() * sizeof(T));
    if (!v.empty()) BCHECK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}

}  // namespace

void build_skeletons_device(Plan& P, const std::vector<std::vector<int64_t>>& leaf_points) {
    Tree& t = P.tree;
    Skel& sk = P.sk;
    const int dim = t.dim;
    const int64_t nb = t.nb;
    sk.cplx = (P.kind == 2 || P.kind == 3);
    const int w = sk.cplx ? 2 : 1;                 // doubles per value
    const size_t sz = sizeof(double) * w;
    std::vector<std::vector<int64_t>> idx(nb), piv(nb);
    std::vector<std::vector<double>> Tb(nb);
    std::vector<int32_t> kk(nb, 0);
    P.t_id_kernels = 0.0;
    P.id_flops = 0.0;

    DBuf d_pts, d_I, d_ptr, d_cen, d_prox, d_off, d_ws, d_k, d_piv, d_Toff, d_T;
    const double* pts = put(d_pts, P.pts);
    cudaEvent_t ev0, ev1;
    BCHECK(cudaEventCreate(&ev0));
    BCHECK(cudaEventCreate(&ev1));
    size_t free_b = 0, total_b = 0;
    BCHECK(cudaMemGetInfo(&free_b, &total_b));
    const size_t ws_cap = std::max<size_t>((size_t)1 << 28, std::min<size_t>((size_t)4 << 30, free_b / 3));

    try {
        for (int l = t.L; l >= 1; --l) {
            const int64_t b0 = t.level_ptr[l], b1 = t.level_ptr[l + 1];
            for (int64_t b = b0; b < b1; ++b) {
                std::vector<int64_t>& I = idx[b];
                if (t.is_leaf[b]) {
                    I = leaf_points[b];
                } else {
                    for (int64_t q = t.child_ptr[b]; q < t.child_ptr[b + 1]; ++q) {
                        const int64_t c = t.child[q];
                        for (int i = 0; i < kk[c]; ++i) I.push_back(idx[c][piv[c][i]]);
                    }
                }
            }
            if (l == 1) {
                for (int64_t b = b0; b < b1; ++b) {
                    piv[b].resize(idx[b].size());
                    std::iota(piv[b].begin(), piv[b].end(), 0);
                    kk[b] = (int32_t)idx[b].size();
                }
                continue;
            }
            const double a = t.side / std::ldexp(1.0, l);
            const double zero3[3] = {0.0, 0.0, 0.0};
            std::vector<double> prox;
            proxy_points(zero3, a, dim, P.proxy_p, prox);
            const int np = (int)(prox.size() / dim);
            const int m = sk.cplx ? 2 * np : np;
            const double* d_prox_p = put(d_prox, prox);

            for (int64_t c0 = b0; c0 < b1;) {
                // a chunk of boxes whose matrices fit the workspace
                int64_t c1 = c0;
                size_t elems = 0;
                int n_max = 0;
                while (c1 < b1) {
                    const size_t e = (size_t)m * idx[c1].size();
                    if (c1 > c0 && (elems + e) * sz > ws_cap) break;
                    elems += e;
                    n_max = std::max(n_max, (int)idx[c1].size());
                    ++c1;
                }
                const int64_t nbox = c1 - c0;
                std::vector<int64_t> hptr(nbox + 1, 0), hoff(nbox), hI;
                std::vector<double> hcen(3 * nbox, 0.0);
                size_t acc = 0;
                for (int64_t i = 0; i < nbox; ++i) {
                    const int64_t b = c0 + i;
                    hptr[i + 1] = hptr[i] + (int64_t)idx[b].size();
                    hoff[i] = (int64_t)acc;
                    acc += (size_t)m * idx[b].size();
                    for (int d = 0; d < dim; ++d)
                        hcen[3 * i + d] = t.corner[d] + ((double)t.coord[b * dim + d] + 0.5) * a;
                }
                hI.reserve(hptr[nbox]);
                for (int64_t i = 0; i < nbox; ++i) hI.insert(hI.end(), idx[c0 + i].begin(), idx[c0 + i].end());

                IdArgs A;
                A.pts = pts;
                A.I = put(d_I, hI);
                A.box_ptr = put(d_ptr, hptr);
                A.cen = put(d_cen, hcen);
                A.prox = d_prox_p;
                A.ws_off = put(d_off, hoff);
                A.ws = d_ws.get(elems * sz);
                A.k_out = (int32_t*)d_k.get(nbox * sizeof(int32_t));
                A.piv_out = (int32_t*)d_piv.get(hptr[nbox] * sizeof(int32_t));
                A.dim = dim;
                A.np = np;
                A.m = m;
                A.n_max = n_max;
                A.kappa = P.kappa;
                A.tol = P.tol;
                const size_t smem = 2 * (size_t)m * sz + (size_t)n_max * sizeof(double);
                if (smem > 200 * 1024) throw Error(-1, "device build: a box is too large for shared memory");
                const bool wide = nbox < 2 * 152;           // fewer boxes than two per SM
                const int nt = wide ? 1024 : kIdThreads;
                void (*kern)(IdArgs) =
                    wide ? (P.kind == 0 ? id_kernel<0, 1024> : P.kind == 1 ? id_kernel<1, 1024>
                            : P.kind == 2 ? id_kernel<2, 1024> : id_kernel<3, 1024>)
                         : (P.kind == 0 ? id_kernel<0, kIdThreads> : P.kind == 1 ? id_kernel<1, kIdThreads>
                            : P.kind == 2 ? id_kernel<2, kIdThreads> : id_kernel<3, kIdThreads>);
                BCHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                BCHECK(cudaEventRecord(ev0));
                kern<<<(unsigned)nbox, nt, smem>>>(A);
                BCHECK(cudaGetLastError());
                BCHECK(cudaEventRecord(ev1));
                std::vector<int32_t> hk(nbox);
                BCHECK(cudaMemcpy(hk.data(), A.k_out, nbox * sizeof(int32_t), cudaMemcpyDeviceToHost));
                float ms = 0.f;
                BCHECK(cudaEventElapsedTime(&ms, ev0, ev1));
                P.t_id_kernels += ms * 1e-3;
                std::vector<int64_t> hTo(nbox + 1, 0);
                for (int64_t i = 0; i < nbox; ++i) {
                    const int64_t n = hptr[i + 1] - hptr[i];
                    const int64_t k = hk[i];
                    if (k < 1 || k > n) throw Error(-5, "device build: non-finite proxy matrix");
                    hTo[i + 1] = hTo[i] + k * (n - k);
                    // flops of the reflector updates (dot, update, norm: 6 per
                    // real element, 4x that for complex)
                    double f = 0.0;
                    for (int64_t j = 0; j < std::min<int64_t>(k, std::min<int64_t>(m, n)); ++j)
                        f += 6.0 * (double)(n - j - 1) * (double)(m - j);
                    P.id_flops += sk.cplx ? 4.0 * f : f;
                }
                const int64_t* dTo = put(d_Toff, hTo);
                void* dT = d_T.get(std::max<int64_t>(hTo[nbox], 1) * sz);
                if (sk.cplx)
                    id_gather_kernel<Zd><<<(unsigned)nbox, kIdThreads>>>((const Zd*)A.ws, A.ws_off, A.box_ptr, m,
                                                                          A.k_out, dTo, (Zd*)dT);
                else
                    id_gather_kernel<double><<<(unsigned)nbox, kIdThreads>>>((const double*)A.ws, A.ws_off,
                                                                              A.box_ptr, m, A.k_out, dTo,
                                                                              (double*)dT);
                BCHECK(cudaGetLastError());
                std::vector<int32_t> hp(hptr[nbox]);
                std::vector<double> hT((size_t)hTo[nbox] * w);
                BCHECK(cudaMemcpy(hp.data(), A.piv_out, hp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
                if (!hT.empty())
                    BCHECK(cudaMemcpy(hT.data(), dT, hT.size() * sizeof(double), cudaMemcpyDeviceToHost));
                for (int64_t i = 0; i < nbox; ++i) {
                    const int64_t b = c0 + i;
                    kk[b] = hk[i];
                    piv[b].assign(hp.begin() + hptr[i], hp.begin() + hptr[i + 1]);
                    Tb[b].assign(hT.begin() + hTo[i] * w, hT.begin() + hTo[i + 1] * w);
                }
                c0 = c1;
            }
        }
    } catch (...) {
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        throw;
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (t.L == 0) {
        idx[0] = leaf_points[0];
        piv[0].resize(idx[0].size());
        std::iota(piv[0].begin(), piv[0].end(), 0);
        kk[0] = (int32_t)idx[0].size();
    }
    store_skeletons(P, idx, piv, Tb, kk);
}

}  // namespace skel
