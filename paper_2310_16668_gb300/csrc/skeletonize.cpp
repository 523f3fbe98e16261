// Algorithm 1 (strong recursive skeletonization) on the host in FP64 /
// complex128.
//
// For every box on levels L..2 (in parallel within a level):
//   I_B  = the leaf's points (ascending) or the children's skeletons
//          concatenated in child order ("slot order");
//   M    = [G(P, I_B); conj(G(P, I_B))] for the proxy points P of Section 2.1
//          (Chebyshev points on the boundary of the box of side 2.95 a centred
//          on B); for real kernels only the first block, which already spans
//          the same column space;
//   column-pivoted Householder QR of M, stopped at the first |R_jj| <=
//          tol |R_00|; S = the first k pivots, R = the rest;
//   T    = R_11^{-1} R_12 (k x |R|), so that M(:,R) ~= M(:,S) T.
// Column norms are recomputed from the updated columns at every step (no
// downdating), which keeps the pivot choice stable near the truncation rank.
// Level-1 boxes keep S = I_B with an empty T: Algorithm 2 never uses a
// level-1 outgoing skeleton charge.
#include <algorithm>
#include <cmath>
#include <numeric>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "host.h"

namespace skel {

namespace {

const double kPi = 3.14159265358979323846;
const double kProxyScale = 2.95;

inline double abs2(double v) { return v * v; }
inline double abs2(const std::complex<double>& v) { return std::norm(v); }
inline double conj_(double v) { return v; }
inline std::complex<double> conj_(const std::complex<double>& v) { return std::conj(v); }

template <class S> S kval(int kind, double kappa, const double* x, const double* y, int dim);
template <> double kval<double>(int kind, double, const double* x, const double* y, int dim) {
    double r2 = 0;
    for (int d = 0; d < dim; ++d) r2 += (x[d] - y[d]) * (x[d] - y[d]);
    if (r2 == 0.0) return 0.0;
    if (kind == 0) return -std::log(std::sqrt(r2)) / (2.0 * kPi);
    return 1.0 / (4.0 * kPi * std::sqrt(r2));
}
template <> std::complex<double> kval<std::complex<double>>(int kind, double kappa, const double* x,
                                                            const double* y, int dim) {
    double r2 = 0;
    for (int d = 0; d < dim; ++d) r2 += (x[d] - y[d]) * (x[d] - y[d]);
    if (r2 == 0.0) return 0.0;
    double r = std::sqrt(r2);
    if (kind == 3) {
        // (i/4) H_0^(1)(kappa r) = (i/4) (J_0 + i Y_0), from the C++17 special functions
        const double kr = kappa * r;
        return std::complex<double>(-0.25 * std::cyl_neumann(0.0, kr), 0.25 * std::cyl_bessel_j(0.0, kr));
    }
    return std::complex<double>(std::cos(kappa * r), std::sin(kappa * r)) / (4.0 * kPi * r);
}

// Column-pivoted Householder QR ID of the column-major m x n matrix M
// (destroyed). Returns piv (S first), k and T (k x (n-k), column-major).
template <class S>
void cpqr_id(std::vector<S>& M, int m, int n, double tol, std::vector<int64_t>& piv, int& k,
             std::vector<S>& T) {
    piv.resize(n);
    std::iota(piv.begin(), piv.end(), 0);
    std::vector<double> nrm(n);
    std::vector<S> rdiag(std::min(m, n));
    for (int c = 0; c < n; ++c) {
        double s = 0;
        const S* col = &M[(size_t)c * m];
        for (int i = 0; i < m; ++i) s += abs2(col[i]);
        nrm[c] = s;
    }
    const int kmax = std::min(m, n);
    double r00 = 0.0;
    k = kmax;
    for (int j = 0; j < kmax; ++j) {
        int p = j;
        for (int c = j + 1; c < n; ++c)
            if (nrm[c] > nrm[p]) p = c;
        const double cn = std::sqrt(nrm[p]);
        if (j == 0) r00 = cn;
        if (j == 0 && cn == 0.0) {   // zero matrix: nothing to compress
            k = n;
            T.clear();
            return;
        }
        if (cn == 0.0 || !(cn > tol * r00)) { k = j; break; }
        if (p != j) {
            std::swap_ranges(M.begin() + (size_t)j * m, M.begin() + (size_t)(j + 1) * m,
                             M.begin() + (size_t)p * m);
            std::swap(piv[j], piv[p]);
            std::swap(nrm[j], nrm[p]);
        }
        S* v = &M[(size_t)j * m];
        const S x0 = v[j];
        const double ax0 = std::sqrt(abs2(x0));
        const S alpha = ax0 == 0.0 ? S(-cn) : S(-(x0 / ax0) * cn);
        v[j] = x0 - alpha;
        double vn2 = 0;
        for (int i = j; i < m; ++i) vn2 += abs2(v[i]);
        rdiag[j] = alpha;
        if (vn2 > 0) {
            for (int c = j + 1; c < n; ++c) {
                S* col = &M[(size_t)c * m];
                S dot = 0;
                for (int i = j; i < m; ++i) dot += conj_(v[i]) * col[i];
                const S f = (2.0 / vn2) * dot;
                double s = 0;
                col[j] -= f * v[j];
                for (int i = j + 1; i < m; ++i) {
                    col[i] -= f * v[i];
                    s += abs2(col[i]);
                }
                nrm[c] = s;
            }
        }
    }
    if (k < 1) k = 1;
    const int r = n - k;
    T.assign((size_t)k * r, S(0));
    for (int c = 0; c < r; ++c) {
        const S* col = &M[(size_t)(k + c) * m];
        S* tc = &T[(size_t)c * k];
        for (int i = k - 1; i >= 0; --i) {
            S acc = col[i];
            for (int s = i + 1; s < k; ++s) acc -= M[(size_t)s * m + i] * tc[s];
            tc[i] = acc / rdiag[i];
        }
    }
}

template <class S>
void skeletonize_all(Plan& P, const std::vector<std::vector<int64_t>>& leaf_points, int nthreads) {
    Tree& t = P.tree;
    Skel& sk = P.sk;
    const int dim = t.dim;
    const int64_t nb = t.nb;
    const int p = P.proxy_p;
    std::vector<std::vector<int64_t>> idx(nb), piv(nb);
    std::vector<std::vector<S>> Tb(nb);
    std::vector<int32_t> kk(nb, 0);
    auto skel_of = [&](int64_t c, std::vector<int64_t>& out) {
        for (int i = 0; i < kk[c]; ++i) out.push_back(idx[c][piv[c][i]]);
    };
    for (int l = t.L; l >= 1; --l) {
        const int64_t b0 = t.level_ptr[l], b1 = t.level_ptr[l + 1];
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
        for (int64_t b = b0; b < b1; ++b) {
            std::vector<int64_t>& I = idx[b];
            if (t.is_leaf[b]) {
                I = leaf_points[b];
            } else {
                for (int64_t q = t.child_ptr[b]; q < t.child_ptr[b + 1]; ++q) skel_of(t.child[q], I);
            }
            const int n = (int)I.size();
            if (l == 1) {
                piv[b].resize(n);
                std::iota(piv[b].begin(), piv[b].end(), 0);
                kk[b] = n;
                continue;
            }
            double a = t.side / std::ldexp(1.0, l), c[3];
            for (int d = 0; d < dim; ++d) c[d] = t.corner[d] + ((double)t.coord[b * dim + d] + 0.5) * a;
            std::vector<double> prox;
            proxy_points(c, a, dim, p, prox);
            const int np = (int)(prox.size() / dim);
            const bool cplx = sk.cplx;
            const int m = cplx ? 2 * np : np;
            std::vector<S> M((size_t)m * n);
            for (int j = 0; j < n; ++j) {
                const double* xj = &P.pts[I[j] * dim];
                for (int i = 0; i < np; ++i) {
                    S g = kval<S>(P.kind, P.kappa, &prox[i * dim], xj, dim);
                    M[(size_t)j * m + i] = g;
                    if (cplx) M[(size_t)j * m + np + i] = conj_(g);
                }
            }
            int k = 0;
            cpqr_id<S>(M, m, n, P.tol, piv[b], k, Tb[b]);
            kk[b] = k;
        }
    }
    if (t.L == 0) {
        idx[0] = leaf_points[0];
        piv[0].resize(idx[0].size());
        std::iota(piv[0].begin(), piv[0].end(), 0);
        kk[0] = (int32_t)idx[0].size();
    }
    std::vector<std::vector<double>> Tw(nb);
    const int w = sk.cplx ? 2 : 1;
    for (int64_t b = 0; b < nb; ++b) {
        const double* src = reinterpret_cast<const double*>(Tb[b].data());
        Tw[b].assign(src, src + Tb[b].size() * w);
    }
    store_skeletons(P, idx, piv, Tw, kk);
}

}  // namespace

void proxy_points(const double* c, double a, int dim, int p, std::vector<double>& out) {
    const double h = 0.5 * kProxyScale * a;
    std::vector<double> t(p);
    for (int k = 1; k <= p; ++k) t[k - 1] = h * std::cos((2.0 * k - 1.0) * kPi / (2.0 * p));
    out.clear();
    if (dim == 2) {
        for (int axis = 0; axis < 2; ++axis)
            for (double sgn : {-1.0, 1.0})
                for (int i = 0; i < p; ++i) {
                    double v[2];
                    v[axis] = sgn * h;
                    v[1 - axis] = t[i];
                    out.push_back(c[0] + v[0]);
                    out.push_back(c[1] + v[1]);
                }
    } else {
        for (int axis = 0; axis < 3; ++axis) {
            int o0 = axis == 0 ? 1 : 0, o1 = axis == 2 ? 1 : 2;
            for (double sgn : {-1.0, 1.0})
                for (int i = 0; i < p; ++i)
                    for (int j = 0; j < p; ++j) {
                        double v[3];
                        v[axis] = sgn * h;
                        v[o0] = t[i];
                        v[o1] = t[j];
                        for (int d = 0; d < 3; ++d) out.push_back(c[d] + v[d]);
                    }
        }
    }
}

// Flatten per-box index sets, pivots, ranks and T blocks (raw doubles:
// complex entries as two) into the plan.
void store_skeletons(Plan& P, const std::vector<std::vector<int64_t>>& idx,
                     const std::vector<std::vector<int64_t>>& piv, const std::vector<std::vector<double>>& Tw,
                     const std::vector<int32_t>& kk) {
    Skel& sk = P.sk;
    const int64_t nb = P.tree.nb;
    const int w = sk.cplx ? 2 : 1;
    sk.idx_ptr.assign(nb + 1, 0);
    sk.T_ptr.assign(nb + 1, 0);
    sk.k = kk;
    for (int64_t b = 0; b < nb; ++b) {
        sk.idx_ptr[b + 1] = sk.idx_ptr[b] + (int64_t)idx[b].size();
        sk.T_ptr[b + 1] = sk.T_ptr[b] + (int64_t)(Tw[b].size() / w);
    }
    sk.idx.resize(sk.idx_ptr[nb]);
    sk.piv.resize(sk.idx_ptr[nb]);
    sk.T.resize((size_t)sk.T_ptr[nb] * w);
    for (int64_t b = 0; b < nb; ++b) {
        std::copy(idx[b].begin(), idx[b].end(), sk.idx.begin() + sk.idx_ptr[b]);
        std::copy(piv[b].begin(), piv[b].end(), sk.piv.begin() + sk.idx_ptr[b]);
        std::copy(Tw[b].begin(), Tw[b].end(), sk.T.begin() + sk.T_ptr[b] * w);
    }
}

std::complex<double> kernel_value(int kind, double kappa, const double* x, const double* y, int dim) {
    if (kind == 2 || kind == 3) return kval<std::complex<double>>(kind, kappa, x, y, dim);
    return kval<double>(kind, kappa, x, y, dim);
}

void build_skeletons(Plan& P, const std::vector<std::vector<int64_t>>& leaf_points, int nthreads) {
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    P.sk.cplx = (P.kind == 2 || P.kind == 3);
    if (P.sk.cplx)
        skeletonize_all<std::complex<double>>(P, leaf_points, nthreads);
    else
        skeletonize_all<double>(P, leaf_points, nthreads);
}

}  // namespace skel
