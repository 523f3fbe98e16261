// extern "C" entry points of skel.h. Every call catches all exceptions and
// turns them into SKEL_ERR_* codes plus a thread-local message.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <unordered_map>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "../../include/skel.h"
#include "device.h"
#include "host.h"

using skel::Error;

struct skel_plan {
    skel::Plan plan;
    skel::DevicePlan* dev = nullptr;
    int nrhs_max = 32;
    bool host_only = false;
    double t_upload = 0;
    int64_t n_items = 0, pairs_direct = 0, pairs_far = 0;
    int64_t n_tc_items = 0, n_tc_tiles = 0, n_mix_items = 0, pairs_tc = 0;
    // skel_merge: a plan over many point sets keeps only the device part and
    // the sets' summed statistics (its host tree and IDs stay with the sets)
    bool merged = false;
    int n_sets = 1;
    skel_stats mstats{};
};

namespace {

thread_local std::string g_err;

double now() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

template <class F>
int guarded(F&& f) {
    try {
        g_err.clear();
        f();
        return SKEL_OK;
    } catch (const Error& e) {
        return fail(e.code, e.what());
    } catch (const std::bad_alloc&) {
        return fail(SKEL_ERR_OOM, "host allocation failed");
    } catch (const std::exception& e) {
        return fail(SKEL_ERR_ARG, e.what());
    } catch (...) {
        return fail(SKEL_ERR_ARG, "unknown error");
    }
}

void check_kernel(skel_kernel k, int dim) {
    const std::string m = skel::kernel_args_error(k.kind, k.kappa, dim);
    if (!m.empty()) throw Error(SKEL_ERR_ARG, m);
}

void check_points(const double* pts, int64_t n, int dim) {
    if (!pts) throw Error(SKEL_ERR_ARG, "points is NULL");
    if (n < 1) throw Error(SKEL_ERR_ARG, "n must be >= 1");
    if (n > ((int64_t)1 << 31) - 1) throw Error(SKEL_ERR_ARG, "n too large");
    for (int64_t i = 0; i < n * dim; ++i)
        if (!std::isfinite(pts[i])) throw Error(SKEL_ERR_NUMERIC, "non-finite point coordinate");
}

void finalize(skel_plan* h, const skel_options* opts) {
    h->nrhs_max = (opts && opts->nrhs_max > 0) ? opts->nrhs_max : 32;
    if (h->nrhs_max > 256) throw Error(SKEL_ERR_ARG, "nrhs_max must be <= 256");
    h->host_only = opts && opts->host_only;
    double t0 = now();
    skel::Layout lay;
    skel::build_layout(h->plan, lay);
    h->n_items = (int64_t)lay.items.size();
    h->pairs_direct = lay.pairs_direct;
    h->pairs_far = lay.pairs_far;
    h->n_tc_items = (int64_t)lay.tc_items.size();
    h->n_tc_tiles = (int64_t)lay.tc_tiles.size();
    h->n_mix_items = (int64_t)lay.mix_items.size();
    h->pairs_tc = lay.pairs_tc;
    if (opts && (opts->store_tiles < 0 || opts->store_tiles > 2)) throw Error(SKEL_ERR_ARG, "store_tiles must be 0, 1 or 2");
    if (opts && opts->store_stages != 0 && opts->store_stages != 4 && opts->store_stages != 5 && opts->store_stages != 8)
        throw Error(SKEL_ERR_ARG, "store_stages must be 0, 4, 5 or 8");
    if (!h->host_only)
        h->dev = skel::device_plan_create(h->plan, lay, h->nrhs_max, opts ? opts->store_tiles : 0,
                                          opts && opts->store_stages ? opts->store_stages : 4,
                                          opts && opts->updown_tc);
    h->t_upload = now() - t0;
}

// device pointer usable on the current device (true), host pointer (false);
// device memory of another device is an argument error
bool is_device_ptr(const void* p) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        throw Error(SKEL_ERR_CUDA, "cudaGetDevice failed");
    }
    const int w = skel::pointer_place(p, dev);
    if (w < 0) throw Error(SKEL_ERR_ARG, "a pointer is device memory of another CUDA device");
    return w == 1;
}

// the device address of page-locked host memory (cudaHostAlloc /
// cudaHostRegister; with unified addressing the same pointer), else null
const void* mapped_host(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int do_apply(skel_handle h, const void* q, void* u, int nrhs, int precision, void* stream, bool transpose) {
    return guarded([&] {
        if (!h) throw Error(SKEL_ERR_ARG, "handle is NULL");
        if (!q || !u) throw Error(SKEL_ERR_ARG, "q or u is NULL");
        if (h->host_only || !h->dev) throw Error(SKEL_ERR_STATE, "plan was built host-only");
        if (nrhs < 1 || nrhs > h->nrhs_max) throw Error(SKEL_ERR_ARG, "nrhs out of range [1, nrhs_max]");
        if (precision != SKEL_FP64 && precision != SKEL_FP32 && precision != SKEL_FP32_TC)
            throw Error(SKEL_ERR_ARG, "unknown precision");
        skel::DevicePlan* dp = h->dev;
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != dp->device) throw Error(SKEL_ERR_STATE, "current CUDA device differs from the plan's device");
        const size_t elem = (precision == SKEL_FP64 ? 8 : 4) * (dp->cplx ? 2 : 1);
        const size_t bytes = elem * (size_t)dp->N * nrhs;
        if (q == u || ((const char*)q < (const char*)u + bytes && (const char*)u < (const char*)q + bytes))
            throw Error(SKEL_ERR_ARG, "q and u overlap");
        bool qd = is_device_ptr(q), ud = is_device_ptr(u);
        const bool host_call = !qd || !ud;
        cudaStream_t st = (cudaStream_t)stream;
        const void* qq = q;
        void* uu = u;
        // page-locked host buffers are read and written in place by the
        // permutation kernels (over the host link): no staging copy
        if (!qd) {
            if (const void* m = mapped_host(q)) qq = m, qd = true;
        }
        if (!ud) {
            if (const void* m = mapped_host(u)) uu = const_cast<void*>(m), ud = true;
        }
        if (!qd || !ud) {
            if (dp->stage_bytes < bytes) {
                cudaFree(dp->stage_in);
                cudaFree(dp->stage_out);
                dp->stage_in = dp->stage_out = nullptr;
                dp->stage_bytes = 0;
                if (skel::alloc_should_fail() || cudaMalloc(&dp->stage_in, bytes) != cudaSuccess ||
                    cudaMalloc(&dp->stage_out, bytes) != cudaSuccess) {
                    cudaGetLastError();
                    cudaFree(dp->stage_in);
                    cudaFree(dp->stage_out);
                    dp->stage_in = dp->stage_out = nullptr;
                    throw Error(SKEL_ERR_OOM, "staging allocation failed");
                }
                dp->stage_bytes = bytes;
            }
            if (!qd) {
                if (cudaMemcpyAsync(dp->stage_in, q, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
                    throw Error(SKEL_ERR_CUDA, "host-to-device copy failed");
                qq = dp->stage_in;
            }
            if (!ud) uu = dp->stage_out;
        }
        skel::device_apply(dp, qq, uu, nrhs, precision, transpose, stream);
        if (!ud) {
            if (cudaMemcpyAsync(u, uu, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
                throw Error(SKEL_ERR_CUDA, "device-to-host copy failed");
        }
        if (host_call) {
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) throw Error(SKEL_ERR_CUDA, std::string("apply: ") + cudaGetErrorString(e));
        }
    });
}

void check_build_args(skel_kernel k, double tol, int leaf_size, const skel_options* opts) {
    if (!(tol > 0 && tol < 1)) throw Error(SKEL_ERR_ARG, "tol must be in (0, 1)");
    if (leaf_size < 1) throw Error(SKEL_ERR_ARG, "leaf_size must be >= 1");
    if (opts && opts->device_build && opts->host_only)
        throw Error(SKEL_ERR_ARG, "device_build needs a device plan (host_only = 0)");
    (void)k;
}

// Tree, neighbor lists and Algorithm 1 of one point set (arguments already
// checked); the device part comes in finalize(). threads: host threads of
// the host ID build (0 = all).
skel_plan* build_host(const double* points, int64_t n, int dim, skel_kernel k, double tol, int leaf_size,
                      const skel_options* opts, int threads) {
    skel_plan* h = new skel_plan();
    try {
        skel::Plan& P = h->plan;
        P.kind = k.kind;
        P.kappa = k.kappa;
        P.tol = tol;
        P.leaf_size = leaf_size;
        P.proxy_p = (opts && opts->proxy_p > 0) ? opts->proxy_p : (dim == 2 ? 32 : 12);
        P.pts.assign(points, points + n * dim);
        double t0 = now();
        std::vector<std::vector<int64_t>> leaf_points;
        skel::build_tree(points, n, dim, leaf_size, P.tree, leaf_points);
        double t1 = now();
        if (opts && opts->device_build) {
            skel::build_skeletons_device(P, leaf_points);
            P.skel_on_device = true;
        } else {
            skel::build_skeletons(P, leaf_points, threads);
        }
        P.t_tree = t1 - t0;
        P.t_skel = now() - t1;
    } catch (...) {
        delete h;
        throw;
    }
    return h;
}

void destroy(skel_plan* h) {
    if (!h) return;
    if (h->dev) skel::device_plan_destroy(h->dev);
    delete h;
}

}  // namespace

namespace skel {
// lets other translation units of the C-ABI report through skel_last_error
int set_error(int code, const std::string& msg) { return fail(code, msg); }

std::string kernel_args_error(int kind, double kappa, int dim) {
    if (kind != SKEL_LAPLACE_2D && kind != SKEL_LAPLACE_3D && kind != SKEL_HELMHOLTZ_3D && kind != SKEL_HELMHOLTZ_2D)
        return "unknown kernel kind";
    const bool two_d = kind == SKEL_LAPLACE_2D || kind == SKEL_HELMHOLTZ_2D;
    if (two_d != (dim == 2) || (dim != 2 && dim != 3))
        return "dim does not match the kernel (2D kernels: dim 2, others: dim 3)";
    if (kind == SKEL_HELMHOLTZ_3D && !(std::isfinite(kappa) && kappa >= 0)) return "kappa must be finite and >= 0";
    if (kind == SKEL_HELMHOLTZ_2D && !(std::isfinite(kappa) && kappa > 0))
        return "kappa must be finite and > 0 for the 2D Helmholtz kernel";
    return "";
}

int pointer_place(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeManaged) return 1;
    if (a.type == cudaMemoryTypeDevice) return a.device == dev ? 1 : -1;
    return 0;
}
}  // namespace skel

extern "C" {

int skel_build(const double* points, int64_t n, int dim, skel_kernel k, double tol, int leaf_size,
               const skel_options* opts, skel_handle* out) {
    return guarded([&] {
        if (!out) throw Error(SKEL_ERR_ARG, "out is NULL");
        check_kernel(k, dim);
        check_points(points, n, dim);
        check_build_args(k, tol, leaf_size, opts);
        skel_plan* h = build_host(points, n, dim, k, tol, leaf_size, opts, opts ? opts->num_threads : 0);
        try {
            finalize(h, opts);
        } catch (...) {
            destroy(h);
            throw;
        }
        *out = h;
    });
}

int skel_build_batch(int nsets, const double* const* points, const int64_t* n, int dim, skel_kernel k, double tol,
                     int leaf_size, const skel_options* opts, skel_handle* out) {
    return guarded([&] {
        if (nsets < 1 || !points || !n || !out) throw Error(SKEL_ERR_ARG, "nsets < 1 or a NULL array");
        check_kernel(k, dim);
        for (int i = 0; i < nsets; ++i) check_points(points[i], n[i], dim);
        check_build_args(k, tol, leaf_size, opts);
        std::vector<skel_plan*> hs(nsets, nullptr);
        // host phases: many small sets in parallel (one thread each), few
        // large ones one after the other with every thread; Algorithm 1 on
        // the GPU always one after the other
        int nthr = 1;
#ifdef _OPENMP
        nthr = (opts && opts->num_threads > 0) ? opts->num_threads : omp_get_max_threads();
#endif
        const bool across = !(opts && opts->device_build) && nsets >= nthr;
        std::vector<int> codes(nsets, SKEL_OK);
        std::vector<std::string> msgs(nsets);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthr) if (across)
        for (int i = 0; i < nsets; ++i) {
            try {
                hs[i] = build_host(points[i], n[i], dim, k, tol, leaf_size, opts, across ? 1 : nthr);
            } catch (const Error& e) {
                codes[i] = e.code;
                msgs[i] = e.what();
            } catch (const std::bad_alloc&) {
                codes[i] = SKEL_ERR_OOM;
                msgs[i] = "host allocation failed";
            } catch (const std::exception& e) {
                codes[i] = SKEL_ERR_ARG;
                msgs[i] = e.what();
            } catch (...) {
                codes[i] = SKEL_ERR_ARG;
                msgs[i] = "unknown error";
            }
        }
        try {
            for (int i = 0; i < nsets; ++i)
                if (codes[i] != SKEL_OK) throw Error(codes[i], "set " + std::to_string(i) + ": " + msgs[i]);
            for (int i = 0; i < nsets; ++i) finalize(hs[i], opts);
        } catch (...) {
            for (skel_plan* h : hs) destroy(h);
            throw;
        }
        for (int i = 0; i < nsets; ++i) out[i] = hs[i];
    });
}

int skel_apply(skel_handle h, const void* q, void* u, int nrhs, int precision, void* stream) {
    return do_apply(h, q, u, nrhs, precision, stream, false);
}

int skel_apply_transpose(skel_handle h, const void* ubar, void* qbar, int nrhs, int precision, void* stream) {
    return do_apply(h, ubar, qbar, nrhs, precision, stream, true);
}

int skel_apply_batch(const skel_handle* hs, int nsets, const void* const* q, void* const* u, int nrhs,
                     int precision, int transpose, void* stream) {
    return guarded([&] {
        if (!hs || !q || !u) throw Error(SKEL_ERR_ARG, "NULL argument");
        if (nsets < 0) throw Error(SKEL_ERR_ARG, "nsets must be >= 0");
        if (precision != SKEL_FP64 && precision != SKEL_FP32 && precision != SKEL_FP32_TC)
            throw Error(SKEL_ERR_ARG, "unknown precision");
        int cur = 0;
        cudaGetDevice(&cur);
        // validate everything before queueing anything
        for (int i = 0; i < nsets; ++i) {
            skel_handle h = hs[i];
            if (!h) throw Error(SKEL_ERR_ARG, "handle " + std::to_string(i) + " is NULL");
            if (h->host_only || !h->dev) throw Error(SKEL_ERR_STATE, "plan " + std::to_string(i) + " is host-only");
            if (h->dev->device != cur) throw Error(SKEL_ERR_STATE, "plan " + std::to_string(i) + " is on another device");
            if (nrhs < 1 || nrhs > h->nrhs_max) throw Error(SKEL_ERR_ARG, "nrhs out of range for plan " + std::to_string(i));
            if (!q[i] || !u[i] || q[i] == u[i]) throw Error(SKEL_ERR_ARG, "bad q / u for plan " + std::to_string(i));
            if (!is_device_ptr(q[i]) || !is_device_ptr(u[i]))
                throw Error(SKEL_ERR_ARG, "skel_apply_batch takes device pointers only (plan " + std::to_string(i) + ")");
        }
        for (int i = 0; i < nsets; ++i)
            skel::device_apply(hs[i]->dev, q[i], u[i], nrhs, precision, transpose != 0, stream);
    });
}

int skel_merge(const skel_handle* hs, int nsets, const skel_options* opts, skel_handle* out) {
    return guarded([&] {
        if (!hs || !out || nsets < 1) throw Error(SKEL_ERR_ARG, "NULL argument or nsets < 1");
        for (int i = 0; i < nsets; ++i) {
            if (!hs[i]) throw Error(SKEL_ERR_ARG, "handle " + std::to_string(i) + " is NULL");
            if (hs[i]->merged) throw Error(SKEL_ERR_ARG, "handle " + std::to_string(i) + " is itself a merged plan");
            const skel::Plan& a = hs[i]->plan;
            const skel::Plan& b = hs[0]->plan;
            if (a.kind != b.kind || a.kappa != b.kappa || a.tree.dim != b.tree.dim)
                throw Error(SKEL_ERR_ARG, "plan " + std::to_string(i) + " has another kernel, kappa or dim");
        }
        const double t0 = now();
        std::vector<skel::Layout> lays(nsets);
        std::vector<int> codes(nsets, SKEL_OK);
        std::vector<std::string> msgs(nsets);
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = 0; i < nsets; ++i) {
            try {
                skel::build_layout(hs[i]->plan, lays[i]);
            } catch (const Error& e) {
                codes[i] = e.code;
                msgs[i] = e.what();
            } catch (const std::bad_alloc&) {
                codes[i] = SKEL_ERR_OOM;
                msgs[i] = "host allocation failed";
            } catch (...) {
                codes[i] = SKEL_ERR_ARG;
                msgs[i] = "layout failed";
            }
        }
        for (int i = 0; i < nsets; ++i)
            if (codes[i] != SKEL_OK) throw Error(codes[i], "set " + std::to_string(i) + ": " + msgs[i]);
        std::vector<const skel::Layout*> lp;
        std::vector<int64_t> np, nb;
        for (int i = 0; i < nsets; ++i) {
            lp.push_back(&lays[i]);
            np.push_back(hs[i]->plan.tree.n);
            nb.push_back(hs[i]->plan.tree.nb);
        }
        const skel::Plan& P0 = hs[0]->plan;
        skel::Layout m;
        skel::merge_layouts(lp, np, nb, P0.sk.cplx ? 2 : 1, m);
        lays.clear();
        skel_plan* h = new skel_plan();
        try {
            h->merged = true;
            h->n_sets = nsets;
            h->plan.kind = P0.kind;
            h->plan.kappa = P0.kappa;
            h->plan.tree.dim = P0.tree.dim;
            h->plan.sk.cplx = P0.sk.cplx;
            skel_stats& st = h->mstats;
            std::memset(&st, 0, sizeof(st));
            st.dim = P0.tree.dim;
            for (int i = 0; i < nsets; ++i) {
                skel_stats si;
                if (skel_info(hs[i], &si) != SKEL_OK) throw Error(SKEL_ERR_ARG, g_err);
                st.n_points += si.n_points;
                st.n_levels = std::max(st.n_levels, si.n_levels);
                st.n_boxes += si.n_boxes;
                st.n_leaves += si.n_leaves;
                st.k_max = std::max(st.k_max, si.k_max);
                st.n_index += si.n_index;
                st.n_T += si.n_T;
                st.n_colleague += si.n_colleague;
                st.n_coarse += si.n_coarse;
                st.n_fine += si.n_fine;
                st.t_tree += si.t_tree;
                st.t_skel += si.t_skel;
                st.t_id_kernels += si.t_id_kernels;
                st.id_gflop += si.id_gflop;
                st.skel_on_device |= si.skel_on_device;
                st.n_proxy = si.n_proxy;
            }
            h->plan.tree.n = st.n_points;
            h->plan.tree.L = st.n_levels;
            st.pairs_direct = h->pairs_direct = m.pairs_direct;
            st.pairs_far = h->pairs_far = m.pairs_far;
            st.n_work_items = h->n_items = (int64_t)m.items.size();
            st.n_tc_items = h->n_tc_items = (int64_t)m.tc_items.size();
            st.n_tc_tiles = h->n_tc_tiles = (int64_t)m.tc_tiles.size();
            st.n_mix_items = h->n_mix_items = (int64_t)m.mix_items.size();
            st.pairs_tc = h->pairs_tc = m.pairs_tc;
            h->nrhs_max = (opts && opts->nrhs_max > 0) ? opts->nrhs_max : 32;
            if (h->nrhs_max > 256) throw Error(SKEL_ERR_ARG, "nrhs_max must be <= 256");
            h->host_only = opts && opts->host_only;
            if (opts && (opts->store_tiles < 0 || opts->store_tiles > 2))
                throw Error(SKEL_ERR_ARG, "store_tiles must be 0, 1 or 2");
            if (opts && opts->store_stages != 0 && opts->store_stages != 4 && opts->store_stages != 5 &&
                opts->store_stages != 8)
                throw Error(SKEL_ERR_ARG, "store_stages must be 0, 4, 5 or 8");
            if (!h->host_only)
                h->dev = skel::device_plan_create(h->plan, m, h->nrhs_max, opts ? opts->store_tiles : 0,
                                                  opts && opts->store_stages ? opts->store_stages : 4,
                                          opts && opts->updown_tc);
            h->t_upload = st.t_upload = now() - t0;
        } catch (...) {
            destroy(h);
            throw;
        }
        *out = h;
    });
}

void skel_free(skel_handle h) {
    if (!h) return;
    skel::device_plan_destroy(h->dev);
    delete h;
}

int skel_info(skel_handle h, skel_stats* s) {
    return guarded([&] {
        if (!h || !s) throw Error(SKEL_ERR_ARG, "NULL argument");
        if (h->merged) {
            *s = h->mstats;
            s->device_bytes = h->dev ? h->dev->bytes : 0;
            s->stored_tile_bytes = h->dev ? h->dev->stored_bytes : 0;
            s->pairs_stored = h->dev ? h->dev->pairs_stored : 0;
            s->store_mode = h->dev ? h->dev->store_mode : 0;
            return;
        }
        const skel::Plan& P = h->plan;
        const skel::Tree& t = P.tree;
        std::memset(s, 0, sizeof(*s));
        s->n_points = t.n;
        s->dim = t.dim;
        s->n_levels = t.L;
        s->n_boxes = t.nb;
        for (int64_t b = 0; b < t.nb; ++b) {
            s->n_leaves += t.is_leaf[b];
            if (t.level[b] >= 2) s->k_max = std::max(s->k_max, (int)P.sk.k[b]);
        }
        s->n_index = P.sk.idx_ptr[t.nb];
        s->n_T = P.sk.T_ptr[t.nb];
        s->n_colleague = (int64_t)t.coll.size();
        s->n_coarse = (int64_t)t.coarse.size();
        s->n_fine = (int64_t)t.fine.size();
        s->pairs_direct = h->pairs_direct;
        s->pairs_far = h->pairs_far;
        s->n_work_items = h->n_items;
        s->t_tree = P.t_tree;
        s->t_skel = P.t_skel;
        s->t_upload = h->t_upload;
        s->device_bytes = h->dev ? h->dev->bytes : 0;
        s->n_tc_items = h->n_tc_items;
        s->n_tc_tiles = h->n_tc_tiles;
        s->n_mix_items = h->n_mix_items;
        s->pairs_tc = h->pairs_tc;
        s->skel_on_device = P.skel_on_device ? 1 : 0;
        s->t_id_kernels = P.t_id_kernels;
        s->id_gflop = P.id_flops * 1e-9;
        s->stored_tile_bytes = h->dev ? h->dev->stored_bytes : 0;
        s->n_proxy = t.dim == 2 ? 4 * P.proxy_p : 6 * P.proxy_p * P.proxy_p;
        s->pairs_stored = h->dev ? h->dev->pairs_stored : 0;
        s->store_mode = h->dev ? h->dev->store_mode : 0;
    });
}

const char* skel_last_error(void) { return g_err.c_str(); }

int skel_plan_get_dims(skel_handle h, skel_plan_dims* d) {
    return guarded([&] {
        if (!h || !d) throw Error(SKEL_ERR_ARG, "NULL argument");
        if (h->merged) throw Error(SKEL_ERR_STATE, "a merged plan has no single tree to export");
        const skel::Plan& P = h->plan;
        std::memset(d, 0, sizeof(*d));
        d->n_boxes = P.tree.nb;
        d->n_index = P.sk.idx_ptr[P.tree.nb];
        d->n_T = P.sk.T_ptr[P.tree.nb];
        d->dim = P.tree.dim;
        d->is_complex = P.sk.cplx ? 1 : 0;
        for (int i = 0; i < P.tree.dim; ++i) d->center[i] = P.tree.center[i];
        d->side = P.tree.side;
    });
}

int skel_plan_export(skel_handle h, int32_t* level, int32_t* coord, int64_t* parent, int8_t* is_leaf,
                     int64_t* idx_ptr, int64_t* idx, int64_t* piv, int32_t* k, int64_t* T_ptr, double* T) {
    return guarded([&] {
        if (!h) throw Error(SKEL_ERR_ARG, "handle is NULL");
        if (h->merged) throw Error(SKEL_ERR_STATE, "a merged plan has no single tree to export");
        const skel::Plan& P = h->plan;
        const skel::Tree& t = P.tree;
        const int64_t nb = t.nb;
        if (level) std::copy(t.level.begin(), t.level.end(), level);
        if (coord) for (int64_t i = 0; i < nb * t.dim; ++i) coord[i] = (int32_t)t.coord[i];
        if (parent) std::copy(t.parent.begin(), t.parent.end(), parent);
        if (is_leaf) std::copy(t.is_leaf.begin(), t.is_leaf.end(), is_leaf);
        if (idx_ptr) std::copy(P.sk.idx_ptr.begin(), P.sk.idx_ptr.end(), idx_ptr);
        if (idx) std::copy(P.sk.idx.begin(), P.sk.idx.end(), idx);
        if (piv) std::copy(P.sk.piv.begin(), P.sk.piv.end(), piv);
        if (k) std::copy(P.sk.k.begin(), P.sk.k.end(), k);
        if (T_ptr) std::copy(P.sk.T_ptr.begin(), P.sk.T_ptr.end(), T_ptr);
        if (T) std::copy(P.sk.T.begin(), P.sk.T.end(), T);
    });
}

int skel_plan_import(const double* points, int64_t n, int dim, skel_kernel kern, const double* center,
                     double side, int64_t nb, const int32_t* level, const int32_t* coord,
                     const int64_t* parent, const int8_t* is_leaf, const int64_t* idx_ptr,
                     const int64_t* idx, const int64_t* piv, const int32_t* kk, const int64_t* T_ptr,
                     const double* T, const skel_options* opts, skel_handle* out) {
    return guarded([&] {
        if (!out) throw Error(SKEL_ERR_ARG, "out is NULL");
        check_kernel(kern, dim);
        check_points(points, n, dim);
        if (!center || !level || !coord || !parent || !is_leaf || !idx_ptr || !idx || !piv || !kk || !T_ptr ||
            (!T && T_ptr[nb] > 0))
            throw Error(SKEL_ERR_ARG, "NULL plan array");
        if (!(side > 0) || !std::isfinite(side) || nb < 1) throw Error(SKEL_ERR_ARG, "bad root box or box count");
        const int D = skel::max_depth(dim);
        skel_plan* h = new skel_plan();
        try {
            skel::Plan& P = h->plan;
            P.kind = kern.kind;
            P.kappa = kern.kappa;
            P.pts.assign(points, points + n * dim);
            skel::Tree& t = P.tree;
            t.dim = dim;
            t.n = n;
            t.side = side;
            for (int d = 0; d < dim; ++d) {
                t.center[d] = center[d];
                t.corner[d] = center[d] - side * 0.5;
            }
            t.nb = nb;
            t.level.assign(level, level + nb);
            t.coord.resize(nb * dim);
            for (int64_t i = 0; i < nb * dim; ++i) t.coord[i] = coord[i];
            t.parent.assign(parent, parent + nb);
            t.is_leaf.assign(is_leaf, is_leaf + nb);
            // structural checks
            if (t.level[0] != 0 || t.parent[0] != -1) throw Error(SKEL_ERR_ARG, "box 0 must be the root");
            std::vector<int64_t> nchild(nb, 0);
            for (int64_t b = 1; b < nb; ++b) {
                const int l = t.level[b];
                if (l < 1 || l > D || l < t.level[b - 1]) throw Error(SKEL_ERR_ARG, "boxes not sorted by level");
                const int64_t p = t.parent[b];
                if (p < 0 || p >= b || t.level[p] != l - 1) throw Error(SKEL_ERR_ARG, "bad parent");
                for (int d = 0; d < dim; ++d) {
                    const int64_t c = t.coord[b * dim + d];
                    if (c < 0 || c >= ((int64_t)1 << l) || (c >> 1) != t.coord[p * dim + d])
                        throw Error(SKEL_ERR_ARG, "box coordinates inconsistent with parent");
                }
                nchild[p]++;
            }
            for (int64_t b = 0; b < nb; ++b)
                if ((nchild[b] == 0) != (t.is_leaf[b] != 0)) throw Error(SKEL_ERR_ARG, "is_leaf inconsistent");
            skel::finish_tree(t);
            // box order within a level: strictly increasing Morton key
            // (finish_tree's lookup would silently merge duplicates)
            for (int64_t b = 1; b < nb; ++b) {
                if (t.level[b] != t.level[b - 1]) continue;
                auto key = [&](int64_t x) {
                    uint64_t kk2 = 0;
                    for (int bit = 0; bit < (dim == 2 ? 32 : 21); ++bit)
                        for (int d = 0; d < dim; ++d)
                            kk2 |= (uint64_t)((t.coord[x * dim + d] >> bit) & 1) << (bit * dim + d);
                    return kk2;
                };
                if (!(key(b - 1) < key(b))) throw Error(SKEL_ERR_ARG, "boxes not in Morton order");
            }
            // 2:1 balance: no leaf touches a box two or more levels finer
            for (int64_t b = 0; b < nb; ++b) {
                if (!t.is_leaf[b]) continue;
                for (int64_t q = t.coll_ptr[b]; q < t.coll_ptr[b + 1]; ++q) {
                    const int64_t c = t.coll[q];
                    if (c == b || t.is_leaf[c]) continue;
                    for (int64_t r = t.child_ptr[c]; r < t.child_ptr[c + 1]; ++r) {
                        const int64_t ch = t.child[r];
                        if (t.is_leaf[ch]) continue;
                        for (int64_t s = t.child_ptr[ch]; s < t.child_ptr[ch + 1]; ++s) {
                            const int64_t g = t.child[s];
                            if (skel::touches(t.level[b], &t.coord[b * dim], t.level[g], &t.coord[g * dim], dim))
                                throw Error(SKEL_ERR_ARG, "plan is not 2:1 balanced");
                        }
                    }
                }
            }
            // index sets and IDs
            skel::Skel& sk = P.sk;
            sk.cplx = kern.kind == SKEL_HELMHOLTZ_3D || kern.kind == SKEL_HELMHOLTZ_2D;
            sk.idx_ptr.assign(idx_ptr, idx_ptr + nb + 1);
            if (sk.idx_ptr[0] != 0) throw Error(SKEL_ERR_ARG, "idx_ptr[0] != 0");
            for (int64_t b = 0; b < nb; ++b)
                if (sk.idx_ptr[b + 1] < sk.idx_ptr[b]) throw Error(SKEL_ERR_ARG, "idx_ptr not monotone");
            const int64_t ni = sk.idx_ptr[nb];
            sk.idx.assign(idx, idx + ni);
            sk.piv.assign(piv, piv + ni);
            sk.k.assign(kk, kk + nb);
            sk.T_ptr.assign(T_ptr, T_ptr + nb + 1);
            const int w = sk.cplx ? 2 : 1;
            sk.T.assign(T, T + sk.T_ptr[nb] * w);
            std::vector<char> seen(n, 0);
            const double scale = std::ldexp(1.0, D);
            for (int64_t b = 0; b < nb; ++b) {
                const int64_t nbI = sk.idx_ptr[b + 1] - sk.idx_ptr[b];
                const int64_t* I = &sk.idx[sk.idx_ptr[b]];
                if (t.level[b] == 0 && t.L > 0) {
                    if (nbI != 0) throw Error(SKEL_ERR_ARG, "root must have an empty index set");
                    continue;
                }
                if (nbI < 1 || nbI > (int64_t)1 << 30) throw Error(SKEL_ERR_ARG, "empty index set");
                if (sk.k[b] < 1 || sk.k[b] > nbI) throw Error(SKEL_ERR_ARG, "k out of range");
                if (sk.T_ptr[b + 1] - sk.T_ptr[b] != (int64_t)sk.k[b] * (nbI - sk.k[b]))
                    throw Error(SKEL_ERR_ARG, "T size does not match k x |R|");
                std::vector<char> pv(nbI, 0);
                for (int64_t i = 0; i < nbI; ++i) {
                    const int64_t pp = sk.piv[sk.idx_ptr[b] + i];
                    if (pp < 0 || pp >= nbI || pv[pp]) throw Error(SKEL_ERR_ARG, "piv is not a permutation");
                    pv[pp] = 1;
                    if (I[i] < 0 || I[i] >= n) throw Error(SKEL_ERR_ARG, "point index out of range");
                }
                if (t.is_leaf[b]) {
                    const int l = t.level[b];
                    for (int64_t i = 0; i < nbI; ++i) {
                        if (seen[I[i]]) throw Error(SKEL_ERR_ARG, "point in two leaves");
                        seen[I[i]] = 1;
                        for (int d = 0; d < dim; ++d) {
                            double tt = (points[I[i] * dim + d] - t.corner[d]) / side;
                            int64_t v = (int64_t)std::floor(tt * scale);
                            v = std::min(std::max(v, (int64_t)0), ((int64_t)1 << D) - 1);
                            if ((v >> (D - l)) != t.coord[b * dim + d])
                                throw Error(SKEL_ERR_ARG, "point outside its leaf box");
                        }
                    }
                } else {
                    int64_t o = 0;
                    for (int64_t q = t.child_ptr[b]; q < t.child_ptr[b + 1]; ++q) {
                        const int64_t c = t.child[q];
                        for (int i = 0; i < sk.k[c]; ++i, ++o) {
                            const int64_t s = sk.idx[sk.idx_ptr[c] + sk.piv[sk.idx_ptr[c] + i]];
                            if (o >= nbI || I[o] != s)
                                throw Error(SKEL_ERR_ARG, "tree-box index set is not its children's skeletons");
                        }
                    }
                    if (o != nbI) throw Error(SKEL_ERR_ARG, "tree-box index set is not its children's skeletons");
                }
            }
            for (int64_t i = 0; i < n; ++i)
                if (!seen[i]) throw Error(SKEL_ERR_ARG, "point in no leaf");
            finalize(h, opts);
        } catch (...) {
            if (h->dev) skel::device_plan_destroy(h->dev);
            delete h;
            throw;
        }
        *out = h;
    });
}

int skel_neighbors_export(skel_handle h, int which, int64_t* ptr, int64_t* list) {
    return guarded([&] {
        if (!h || !ptr) throw Error(SKEL_ERR_ARG, "NULL argument");
        if (h->merged) throw Error(SKEL_ERR_STATE, "a merged plan has no single tree to export");
        const skel::Tree& t = h->plan.tree;
        const std::vector<int64_t>* p = nullptr;
        const std::vector<int64_t>* l = nullptr;
        if (which == 0) { p = &t.coll_ptr; l = &t.coll; }
        else if (which == 1) { p = &t.coarse_ptr; l = &t.coarse; }
        else if (which == 2) { p = &t.fine_ptr; l = &t.fine; }
        else throw Error(SKEL_ERR_ARG, "which must be 0, 1 or 2");
        std::copy(p->begin(), p->end(), ptr);
        if (list) std::copy(l->begin(), l->end(), list);
    });
}

int skel_set_profiling(skel_handle h, int max_applies) {
    return guarded([&] {
        if (!h) throw Error(SKEL_ERR_ARG, "handle is NULL");
        if (!h->dev) throw Error(SKEL_ERR_STATE, "plan was built host-only");
        skel::device_set_profiling(h->dev, max_applies);
    });
}

int skel_last_timings(skel_handle h, skel_timings* t) {
    return guarded([&] {
        if (!h || !t) throw Error(SKEL_ERR_ARG, "NULL argument");
        if (!h->dev) throw Error(SKEL_ERR_STATE, "plan was built host-only");
        skel::device_last_timings(h->dev, t->ms, &t->launches, &t->n_applies, &t->ms_main, &t->main_launches);
    });
}

int skel_device_status(skel_handle h) {
    int code = SKEL_OK;
    int rc = guarded([&] {
        if (!h) throw Error(SKEL_ERR_ARG, "handle is NULL");
        if (!h->dev) throw Error(SKEL_ERR_STATE, "plan was built host-only");
        if (skel::device_status(h->dev) != 0) code = SKEL_ERR_TIMEOUT;
    });
    if (rc != SKEL_OK) return rc;
    if (code != SKEL_OK) return fail(code, "a bounded device wait gave up during an earlier apply");
    return SKEL_OK;
}

int skel_test_withhold_tile(skel_handle h, double wait_limit_ms) {
    return guarded([&] {
        if (!h) throw Error(SKEL_ERR_ARG, "handle is NULL");
        if (!h->dev) throw Error(SKEL_ERR_STATE, "plan was built host-only");
        if (!(wait_limit_ms > 0 && wait_limit_ms <= 2000)) throw Error(SKEL_ERR_ARG, "wait_limit_ms must be in (0, 2000]");
        if ((h->dev->cplx && h->dev->kind != SKEL_HELMHOLTZ_3D) || h->dev->n_tc == 0)
            throw Error(SKEL_ERR_STATE, "the plan has no tensor-core items");
        h->dev->test_wait_ns = (uint64_t)(wait_limit_ms * 1e6);
        h->dev->test_withhold = true;
    });
}

int skel_test_fail_alloc(int countdown) {
    return guarded([&] {
        if (countdown < 0) throw Error(SKEL_ERR_ARG, "countdown must be >= 0");
        skel::set_alloc_failure(countdown);
    });
}

int skel_test_set_updown(skel_handle h, int code) {
    return guarded([&] {
        if (!h) throw Error(SKEL_ERR_ARG, "handle is NULL");
        if (!h->dev) throw Error(SKEL_ERR_STATE, "plan was built host-only");
        static const int ok[] = {0, 1, 2, 4, 8, 17, 18, 20, 24};
        bool valid = false;
        for (int c : ok) valid |= c == code;
        if (!valid) throw Error(SKEL_ERR_ARG, "code must be 0, 1, 2, 4, 8, 17, 18, 20 or 24");
        const int nl = (int)h->dev->up_level_ptr.size() - 1;
        h->dev->ud_warps_up.assign(std::max(nl, 0), (int8_t)code);
        h->dev->ud_warps_down.assign(std::max(nl, 0), (int8_t)code);
    });
}

int skel_autotune(skel_handle h, int nrhs, int allow_store, void* stream, skel_tuning* out) {
    return guarded([&] {
        if (!h) throw Error(SKEL_ERR_ARG, "handle is NULL");
        if (!h->dev) throw Error(SKEL_ERR_STATE, "plan was built host-only");
        if (h->dev->cplx) throw Error(SKEL_ERR_ARG, "autotune covers the real kernels");
        if (nrhs < 1 || nrhs > h->nrhs_max) throw Error(SKEL_ERR_ARG, "nrhs must be in [1, nrhs_max]");
        const skel::TuneReport r = skel::device_autotune(h->dev, nrhs, allow_store != 0, stream);
        if (out) {
            out->ms_onfly = r.ms_onfly;
            out->ms_stored = r.ms_stored;
            out->stored = r.stored;
            out->n_updown = r.n_levels;
            out->n_changed = r.n_changed;
            out->ms_updown_default = r.ms_updown_default;
            out->ms_updown_tuned = r.ms_updown_tuned;
            out->tc_stages = r.tc_stages;
            out->ms_sym = r.ms_sym;
            out->tcs_stages = r.tcs_stages;
        }
    });
}

}  // extern "C"
