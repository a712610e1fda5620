// C ABI of libibem (declared in include/ibem.h): handle life cycle, host-side
// tables (Bezier extraction, Bernstein values, FMM transfer matrices) and the
// thin argument checks around the kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include <algorithm>

#include "ibem_internal.cuh"

using namespace ibem;

static thread_local std::string g_last_error;

namespace {

ibem_status fail(ibem_handle* h, ibem_status s, const std::string& msg) {
    if (h) h->err = msg; else g_last_error = msg;
    return s;
}

ibem_status cuda_fail(ibem_handle* h, cudaError_t e, const char* where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? IBEM_ERR_OOM : IBEM_ERR_CUDA, msg);
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& src, cudaStream_t st) {
    size_t n = src.empty() ? 1 : src.size();
    cudaError_t e = cudaMalloc(dst, n * sizeof(T));
    if (e) return e;
    if (!src.empty()) e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    return e;
}

// Solve the (p+1) x (p+1) system V c = rhs with partial pivoting (in place).
void small_solve(int n, std::vector<double> V, std::vector<double>& rhs) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(V[r * n + c]) > std::fabs(V[piv * n + c])) piv = r;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(V[c * n + k], V[piv * n + k]);
            std::swap(rhs[c], rhs[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            double f = V[r * n + c] / V[c * n + c];
            for (int k = c; k < n; ++k) V[r * n + k] -= f * V[c * n + k];
            rhs[r] -= f * rhs[c];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        double s = rhs[c];
        for (int k = c + 1; k < n; ++k) s -= V[c * n + k] * rhs[k];
        rhs[c] = s / V[c * n + c];
    }
}

// Bezier extraction of the uniform p-open knot vector Xi_{p,m} (Sec. 4.3): on
// element ix, b_{ix+r}(x(t)) = sum_i ext[ix][r][i] B_{i,p}(t), found by
// interpolation at p+1 interior points of the element.
std::vector<double> bezier_extraction(int p, int m) {
    int pp = p + 1, ne1 = 1 << m;
    std::vector<double> knots;
    for (int i = 0; i < pp; ++i) knots.push_back(0.0);
    for (int i = 1; i < ne1; ++i) knots.push_back((double)i / ne1);
    for (int i = 0; i < pp; ++i) knots.push_back(1.0);
    std::vector<double> ext((size_t)ne1 * pp * pp);
    std::vector<double> V(pp * pp), B(pp), val(IBEM_MAX_DEG + 1), der(IBEM_MAX_DEG + 1);
    std::vector<std::vector<double>> rhs(pp, std::vector<double>(pp));
    for (int ix = 0; ix < ne1; ++ix) {
        for (int k = 0; k < pp; ++k) {
            double t = (k + 0.5) / pp;
            bernstein(p, t, B.data());
            for (int i = 0; i < pp; ++i) V[k * pp + i] = B[i];
            if (p == 0) {
                rhs[0][k] = 1.0;
                continue;
            }
            local_bsplines(knots.data(), p, ix + p, (ix + t) / ne1, val.data(), der.data());
            for (int r = 0; r < pp; ++r) rhs[r][k] = val[r];
        }
        for (int r = 0; r < pp; ++r) {
            std::vector<double> c = rhs[r];
            small_solve(pp, V, c);
            for (int i = 0; i < pp; ++i) ext[((size_t)ix * pp + r) * pp + i] = c[i];
        }
    }
    return ext;
}

void free_handle(ibem_handle* h) {
    void* ptrs[] = {h->d_patches, h->d_knots, h->d_cpw, h->d_ext, h->d_qgeo, h->d_igeo, h->d_igeo32, h->d_phi,
                    h->d_phi_sub, h->d_rule[0], h->d_rule[1], h->d_rule[2], h->d_M, h->d_S, h->d_balls, h->d_mu1d, h->d_mu1d_off, h->d_near_ptr,
                    h->d_near_src, h->d_near_tgt, h->d_near_cls, h->d_near_orient, h->d_pairs_by_cls[0],
                    h->d_pairs_by_cls[1], h->d_pairs_by_cls[2], h->d_pairs_by_cls[3], h->d_pairs_by_cls[4],
                    h->d_near, h->d_near32, h->d_far_ptr, h->d_far_src, h->d_far_tgt, h->d_K, h->d_Kdf, h->d_xh2, h->d_far_rows,
                    h->d_xs, h->d_ys, h->d_xh, h->d_yh, h->d_xs32, h->d_ys32, h->d_yh32, h->d_src32, h->d_diag,
                    h->d_solver, h->d_red, h->d_status, h->d_Kc, h->d_xh4, h->d_hsx, h->d_hsy,
                    h->d_bj_ptr, h->d_bj_off, h->d_bj_dofs, h->d_bj_inv, h->d_up_ptr, h->d_up_src,
                    h->d_up_tgt, h->d_up_rows, h->d_tr_ptr, h->d_tr_blk, h->d_colpart, h->d_mr, h->d_Mf, h->d_Sf,
                    h->d_gen_pts, h->d_gen_trig, h->d_gen_x, h->d_Kbf, h->d_graded_pairs, h->d_graded_tab,
                    h->d_sl};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->h_red) cudaFreeHost(h->h_red);
    for (auto ev : h->ev_free) cudaEventDestroy(ev);
    for (auto& u : h->ev_used) { cudaEventDestroy(u.second.first); cudaEventDestroy(u.second.second); }
    h->ev_free.clear();
    h->ev_used.clear();
}

ibem_status check_ready(ibem_handle* h) {
    if (!h) return fail(nullptr, IBEM_ERR_ARG, "null handle");
    if (!h->assembled) return fail(h, IBEM_ERR_STATE, "call ibem_assemble first");
    return IBEM_OK;
}

cudaError_t set_device(ibem_handle* h) { return cudaSetDevice(h->device); }

// Errors of the patch description and the mesh topology (IBEM_ERR_GEOMETRY)
// against errors of the parameters (IBEM_ERR_ARG), by the text build_plan returns.
ibem_status plan_error_status(const std::string& msg) {
    if (msg.rfind("null", 0) == 0) return IBEM_ERR_ARG;
    for (const char* key : {"NURBS", "knot", "sphere", "patch", "degenerate", "touching"})
        if (msg.find(key) != std::string::npos) return IBEM_ERR_GEOMETRY;
    return IBEM_ERR_ARG;
}

// the FP64 operator needs stored coupling matrices for Laplace (Helmholtz can
// generate them on the fly)
bool fp64_available(const ibem_handle* h) {
    if (h->P.prm.fp64_coupling == IBEM_COUPLING_FP32_ONLY) return false;
    return h->helm || h->P.n_far == 0 || h->d_K || h->d_Kdf;
}

}  // namespace

extern "C" {

const char* ibem_status_string(ibem_status s) {
    switch (s) {
        case IBEM_OK: return "IBEM_OK";
        case IBEM_ERR_ARG: return "IBEM_ERR_ARG";
        case IBEM_ERR_GEOMETRY: return "IBEM_ERR_GEOMETRY";
        case IBEM_ERR_CUDA: return "IBEM_ERR_CUDA";
        case IBEM_ERR_OOM: return "IBEM_ERR_OOM";
        case IBEM_ERR_NOCONV: return "IBEM_ERR_NOCONV";
        case IBEM_ERR_BREAKDOWN: return "IBEM_ERR_BREAKDOWN";
        case IBEM_ERR_STATE: return "IBEM_ERR_STATE";
    }
    return "IBEM_UNKNOWN";
}

const char* ibem_last_error(const ibem_handle* h) { return h ? h->err.c_str() : g_last_error.c_str(); }

ibem_status ibem_block_tree(const ibem_patch* patches, int npatch, const ibem_params* params, int64_t* n_near,
                            int32_t* near, int64_t* n_far, int32_t* far) {
    if (!n_near || !n_far) return fail(nullptr, IBEM_ERR_ARG, "n_near / n_far must be non-null");
    Plan P;
    std::string msg;
    try {
        msg = build_plan(patches, npatch, params, P);
    } catch (const std::bad_alloc&) {
        return fail(nullptr, IBEM_ERR_OOM, "host allocation failed");
    }
    if (!msg.empty()) return fail(nullptr, plan_error_status(msg), msg);
    *n_near = P.n_near;
    *n_far = P.n_far;
    if (near) {
        for (int64_t e = 0; e < P.E; ++e)
            for (int64_t k = P.near_ptr[e]; k < P.near_ptr[e + 1]; ++k) {
                int pt, xt, yt, ps, xs, ys;
                element_of(P, e, &pt, &xt, &yt);
                element_of(P, P.near_src[k], &ps, &xs, &ys);
                int32_t* o = near + 8 * k;
                o[0] = pt; o[1] = xt; o[2] = yt; o[3] = ps; o[4] = xs; o[5] = ys;
                o[6] = P.near_cls[k]; o[7] = P.near_orient[k];
            }
    }
    if (far) {
        for (int64_t c = 0; c < P.C; ++c)
            for (int64_t k = P.far_ptr[c]; k < P.far_ptr[c + 1]; ++k) {
                int32_t* o = far + 8 * k;
                int a, b, x, y;
                cluster_of(P, c, &a, &b, &x, &y);
                o[0] = a; o[1] = b; o[2] = x; o[3] = y;
                cluster_of(P, P.far_src[k], &a, &b, &x, &y);
                o[4] = a; o[5] = b; o[6] = x; o[7] = y;
            }
    }
    return IBEM_OK;
}

ibem_status ibem_near_orders(const ibem_patch* patches, int npatch, const ibem_params* params, int64_t* n_near,
                             int32_t* order) {
    if (!n_near) return fail(nullptr, IBEM_ERR_ARG, "n_near must be non-null");
    Plan P;
    std::string msg;
    try {
        msg = build_plan(patches, npatch, params, P);
    } catch (const std::bad_alloc&) {
        return fail(nullptr, IBEM_ERR_OOM, "host allocation failed");
    }
    if (!msg.empty()) return fail(nullptr, plan_error_status(msg), msg);
    *n_near = P.n_near;
    if (order) std::copy(P.near_order.begin(), P.near_order.end(), order);
    return IBEM_OK;
}

ibem_status ibem_create(const ibem_patch* patches, int npatch, const ibem_params* params, void* cuda_stream,
                        ibem_handle** out) {
    if (!out) return fail(nullptr, IBEM_ERR_ARG, "out must be non-null");
    *out = nullptr;
    ibem_handle* h = new (std::nothrow) ibem_handle();
    if (!h) return fail(nullptr, IBEM_ERR_OOM, "host allocation failed");
    std::string msg;
    try {
        msg = build_plan(patches, npatch, params, h->P);
    } catch (const std::bad_alloc&) {
        delete h;
        return fail(nullptr, IBEM_ERR_OOM, "host allocation failed");
    }
    if (!msg.empty()) {
        delete h;
        return fail(nullptr, plan_error_status(msg), msg);
    }
    Plan& P = h->P;
    h->helm = params->kernel == IBEM_HELMHOLTZ;
    h->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e) { delete h; return cuda_fail(nullptr, e, "cudaGetDevice"); }
    cudaStream_t st = h->stream;
#define TRY(x, where)                                      \
    do {                                                   \
        cudaError_t _e = (x);                              \
        if (_e) {                                          \
            ibem_status _s = cuda_fail(nullptr, _e, where); \
            free_handle(h);                                \
            delete h;                                      \
            return _s;                                     \
        }                                                  \
    } while (0)
    TRY(upload(&h->d_patches, P.patches, st), "upload patches");
    TRY(upload(&h->d_knots, P.knots, st), "upload knots");
    TRY(upload(&h->d_cpw, P.cpw, st), "upload control points");
    std::vector<double> ext = bezier_extraction(P.p, P.m);
    TRY(upload(&h->d_ext, ext, st), "upload extraction");

    // Bernstein products at the regular and the subdivided Gauss points
    std::vector<double> gx, gw;
    gauss_legendre(P.Q, gx, gw);
    int QQ = P.Q * P.Q, nb = P.nb, pp = P.pp;
    std::vector<double> phi((size_t)QQ * nb), phis((size_t)4 * QQ * nb);
    double bu[IBEM_MAX_P + 1], bv[IBEM_MAX_P + 1];
    for (int sub = -1; sub < 4; ++sub)
        for (int g = 0; g < QQ; ++g) {
            double s = gx[g % P.Q], t = gx[g / P.Q];
            if (sub >= 0) { s = 0.5 * (sub & 1) + 0.5 * s; t = 0.5 * (sub >> 1) + 0.5 * t; }
            bernstein(P.p, s, bu);
            bernstein(P.p, t, bv);
            for (int iv = 0; iv < pp; ++iv)
                for (int iu = 0; iu < pp; ++iu) {
                    double v = bu[iu] * bv[iv];
                    if (sub < 0) phi[(size_t)g * nb + iv * pp + iu] = v;
                    else phis[((size_t)sub * QQ + g) * nb + iv * pp + iu] = v;
                }
        }
    TRY(upload(&h->d_phi, phi, st), "upload phi");
    TRY(upload(&h->d_phi_sub, phis, st), "upload phi_sub");
    for (int c = 0; c < 3; ++c) {
        if (P.n_cls[c] == 0) continue;
        std::vector<double> soa;
        singular_rule(c, P.Qs, soa);
        h->rule_n[c] = (int)(soa.size() / 5);
        TRY(upload(&h->d_rule[c], soa, st), "upload singular rule");
    }

    // FMM transfer matrices (1D): leaf moments and M2M re-expansion
    if (P.q > 0) {
        std::vector<double> z, L(P.q);
        chebyshev_nodes(P.q, z);
        int ng = (P.q + P.p + 1) / 2 + 1;
        std::vector<double> mx, mw;
        gauss_legendre(ng, mx, mw);
        std::vector<double> M((size_t)P.q * pp, 0.0), S((size_t)2 * P.q * P.q);
        double h1 = 1.0 / P.ne1;
        for (int k = 0; k < ng; ++k) {
            lagrange_values(z, mx[k], L.data());
            bernstein(P.p, mx[k], bu);
            for (int a = 0; a < P.q; ++a)
                for (int i = 0; i < pp; ++i) M[a * pp + i] += mw[k] * h1 * L[a] * bu[i];
        }
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < P.q; ++b) {
                lagrange_values(z, 0.5 * (c + z[b]), L.data());
                for (int a = 0; a < P.q; ++a) S[((size_t)c * P.q + a) * P.q + b] = L[a];
            }
        TRY(upload(&h->d_M, M, st), "upload M");
        TRY(upload(&h->d_S, S, st), "upload S");
        TRY(upload(&h->d_balls, P.balls, st), "upload cluster balls");
        std::vector<float> Mf(M.begin(), M.end()), Sf(S.begin(), S.end());
        TRY(upload(&h->d_Mf, Mf, st), "upload Mf");
        TRY(upload(&h->d_Sf, Sf, st), "upload Sf");
    }

    // near and far lists
    std::vector<int32_t> ntgt(P.n_near);
    std::vector<std::vector<int32_t>> bycls(5);
    std::vector<std::vector<int32_t>> bygrade(2 * (IBEM_MAX_GAUSS + 1));   // [subdiv][order]
    for (int64_t t = 0; t < P.E; ++t)
        for (int64_t k = P.near_ptr[t]; k < P.near_ptr[t + 1]; ++k) {
            ntgt[k] = (int32_t)t;
            const int c = P.near_cls[k];
            if ((c == CLS_REGULAR || c == CLS_SUBDIV) && P.near_order[k] != P.Q)
                bygrade[(c == CLS_SUBDIV) * (IBEM_MAX_GAUSS + 1) + P.near_order[k]].push_back((int32_t)k);
            else
                bycls[c].push_back((int32_t)k);
        }
    // graded groups: pairs, Gauss rule and Bernstein products at that order
    {
        std::vector<int32_t> gp;
        std::vector<double> tab;
        for (int sd = 0; sd < 2; ++sd)
            for (int n = 1; n <= IBEM_MAX_GAUSS; ++n) {
                const auto& lst = bygrade[sd * (IBEM_MAX_GAUSS + 1) + n];
                if (lst.empty()) continue;
                ibem_handle::GradedGroup gr{sd ? CLS_SUBDIV : CLS_REGULAR, n, (int64_t)gp.size(),
                                            (int64_t)lst.size(), tab.size()};
                gp.insert(gp.end(), lst.begin(), lst.end());
                std::vector<double> nx, nw;
                gauss_legendre(n, nx, nw);
                tab.insert(tab.end(), nx.begin(), nx.end());
                tab.insert(tab.end(), nw.begin(), nw.end());
                const int nn = n * n, nsub = sd ? 4 : 1;
                for (int sub = 0; sub < nsub; ++sub)
                    for (int g = 0; g < nn; ++g) {
                        double su = nx[g % n], sv = nx[g / n];
                        if (sd) { su = 0.5 * (sub & 1) + 0.5 * su; sv = 0.5 * (sub >> 1) + 0.5 * sv; }
                        bernstein(P.p, su, bu);
                        bernstein(P.p, sv, bv);
                        for (int iv = 0; iv < pp; ++iv)
                            for (int iu = 0; iu < pp; ++iu) tab.push_back(bu[iu] * bv[iv]);
                    }
                h->graded.push_back(gr);
            }
        if (!gp.empty()) {
            TRY(upload(&h->d_graded_pairs, gp, st), "upload graded pairs");
            TRY(upload(&h->d_graded_tab, tab, st), "upload graded rules");
        }
    }
    TRY(upload(&h->d_near_ptr, P.near_ptr, st), "upload near ptr");
    TRY(upload(&h->d_near_src, P.near_src, st), "upload near src");
    TRY(upload(&h->d_near_tgt, ntgt, st), "upload near tgt");
    TRY(upload(&h->d_near_cls, P.near_cls, st), "upload near cls");
    TRY(upload(&h->d_near_orient, P.near_orient, st), "upload near orient");
    for (int c = 0; c < 5; ++c) {
        h->n_list[c] = (int64_t)bycls[c].size();
        TRY(upload(&h->d_pairs_by_cls[c], bycls[c], st), "upload class lists");
    }
    std::vector<int32_t> ftgt(P.n_far);
    for (int64_t c = 0; c < P.C; ++c) {
        if (P.far_ptr[c + 1] > P.far_ptr[c]) h->far_rows.push_back((int32_t)c);
        if (P.far_ptr[c + 1] - P.far_ptr[c] > h->max_far_row) h->max_far_row = (int)(P.far_ptr[c + 1] - P.far_ptr[c]);
        for (int64_t k = P.far_ptr[c]; k < P.far_ptr[c + 1]; ++k) ftgt[k] = (int32_t)c;
    }
    TRY(upload(&h->d_far_ptr, P.far_ptr, st), "upload far ptr");
    // bound on the distance of two interpolation points of a far block, from the
    // cluster balls (the range of the phase kappa r of the coupling)
    for (int64_t c = 0; c < P.C; ++c)
        for (int64_t k = P.far_ptr[c]; k < P.far_ptr[c + 1]; ++k) {
            const double* bi = &P.balls[4 * c];
            const double* bj = &P.balls[4 * (int64_t)P.far_src[k]];
            const double dx = bi[0] - bj[0], dy = bi[1] - bj[1], dz = bi[2] - bj[2];
            h->far_diam = std::max(h->far_diam, std::sqrt(dx * dx + dy * dy + dz * dz) + bi[3] + bj[3]);
        }
    TRY(upload(&h->d_far_src, P.far_src, st), "upload far src");
    TRY(upload(&h->d_far_tgt, ftgt, st), "upload far tgt");
    TRY(upload(&h->d_far_rows, h->far_rows, st), "upload far rows");
    {
        std::vector<int64_t> uptr(P.C + 1, 0);
        std::vector<int32_t> usrc, utgt;
        for (int64_t c = 0; c < P.C; ++c) {
            for (int64_t k = P.far_ptr[c]; k < P.far_ptr[c + 1]; ++k)
                if (P.far_src[k] > c) {
                    usrc.push_back(P.far_src[k]);
                    utgt.push_back((int32_t)c);
                }
            uptr[c + 1] = (int64_t)usrc.size();
            int len = (int)(uptr[c + 1] - uptr[c]);
            if (len > 0) h->up_rows.push_back((int32_t)c);
            if (len > h->max_up_row) h->max_up_row = len;
        }
        // longest rows first: the CTAs of the coupling launch start in this
        // order, so the last wave holds the short rows (smaller tail)
        std::stable_sort(h->up_rows.begin(), h->up_rows.end(), [&](int32_t x, int32_t y) {
            return uptr[x + 1] - uptr[x] > uptr[y + 1] - uptr[y];
        });
        h->n_up = (int64_t)usrc.size();
        std::vector<int64_t> tptr(P.C + 1, 0);
        for (int32_t v : usrc) tptr[v + 1]++;
        for (int64_t c = 0; c < P.C; ++c) tptr[c + 1] += tptr[c];
        std::vector<int32_t> tblk(usrc.size());
        std::vector<int64_t> fill(tptr.begin(), tptr.end() - 1);
        for (int64_t k = 0; k < (int64_t)usrc.size(); ++k) tblk[fill[usrc[k]]++] = (int32_t)k;
        TRY(upload(&h->d_tr_ptr, tptr, st), "upload transposed ptr");
        TRY(upload(&h->d_tr_blk, tblk, st), "upload transposed list");
        TRY(upload(&h->d_up_ptr, uptr, st), "upload upper far ptr");
        TRY(upload(&h->d_up_src, usrc, st), "upload upper far src");
        TRY(upload(&h->d_up_tgt, utgt, st), "upload upper far tgt");
        TRY(upload(&h->d_up_rows, h->up_rows, st), "upload upper far rows");
    }
    h->kpt = (P.q2 + 3) / 4;

    TRY(cudaMalloc(&h->d_qgeo, (size_t)P.nq * 4 * sizeof(double)), "alloc qgeo");
    if (P.q > 0) {
        TRY(cudaMalloc(&h->d_igeo, (size_t)P.C * P.q2 * 4 * sizeof(double)), "alloc igeo");
        TRY(cudaMalloc(&h->d_igeo32, (size_t)P.C * P.q2 * 4 * sizeof(float)), "alloc igeo32");
    }
    TRY(cudaMalloc(&h->d_diag, (size_t)P.N * (h->helm ? 2 : 1) * sizeof(double)), "alloc diag");
    TRY(cudaMalloc(&h->d_red, 64 * sizeof(double)), "alloc red");
    TRY(cudaMalloc(&h->d_status, sizeof(int)), "alloc status");
    TRY(cudaMemsetAsync(h->d_status, 0, sizeof(int), st), "clear status");
    TRY(cudaMallocHost(&h->h_red, 64 * sizeof(double)), "alloc pinned");
    TRY(launch_geometry_tables(h), "geometry tables");
    TRY(cudaStreamSynchronize(st), "create sync");
#undef TRY
    *out = h;
    return IBEM_OK;
}

ibem_status ibem_destroy(ibem_handle* h) {
    if (!h) return IBEM_OK;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    free_handle(h);
    delete h;
    return IBEM_OK;
}

ibem_status ibem_get_info(const ibem_handle* h, ibem_info* info) {
    if (!h || !info) return fail(nullptr, IBEM_ERR_ARG, "null handle or info");
    const Plan& P = h->P;
    info->ndof = P.N;
    info->ndof_super = P.Nstar;
    info->n_elements = P.E;
    info->n_clusters = P.C;
    info->n_quad_points = P.nq;
    info->n_near = P.n_near;
    info->n_far = P.n_far;
    info->n_near_singular[0] = P.n_cls[CLS_IDENTICAL];
    info->n_near_singular[1] = P.n_cls[CLS_EDGE];
    info->n_near_singular[2] = P.n_cls[CLS_VERTEX];
    info->n_near_singular[3] = P.n_cls[CLS_SUBDIV];
    info->bytes_near = P.n_near * (int64_t)P.nb * P.nb * (h->helm ? 16 : 8);
    // the FP64 coupling matrices actually stored: upper half in double-float
    // (Laplace), every far block natively (Laplace) or in double-float (Helmholtz)
    const int64_t per = (int64_t)h->kpt * 4 * P.q2;
    info->bytes_far = h->d_Kdf ? h->n_up * per * 8 : (h->d_K ? P.n_far * per * 8 : (h->d_Kc ? P.n_far * per * 16 : 0));
    info->assembled = h->assembled ? 1 : 0;
    info->max_gauss_order = P.max_order;
    info->n_near_graded = P.n_graded;
    info->stored_ring_depth = h->st_nst;
    return IBEM_OK;
}

// BF16 coupling of the tensor-core path (16 KB per far block), generated on
// the device, if it fits in half of the free memory (IBEM_ERR_OOM otherwise).
static ibem_status store_bf16_coupling(ibem_handle* h) {
    const size_t kb = (size_t)h->P.n_far * 128 * 64 * 2;
    size_t free_b = 0, total_b = 0;
    cudaError_t e;
    if ((e = cudaMemGetInfo(&free_b, &total_b))) return cuda_fail(h, e, "cudaMemGetInfo");
    if (kb > free_b / 2) return fail(h, IBEM_ERR_OOM, "stored BF16 coupling exceeds half of the free device memory");
    if ((e = cudaMalloc(&h->d_Kbf, kb))) {
        h->d_Kbf = nullptr;
        return cuda_fail(h, e, "alloc BF16 coupling");
    }
    if ((e = mr_store_coupling(h)) || (e = cudaStreamSynchronize(h->stream))) {
        cudaFree(h->d_Kbf);
        h->d_Kbf = nullptr;
        return cuda_fail(h, e, "BF16 coupling");
    }
    return IBEM_OK;
}

ibem_status ibem_assemble(ibem_handle* h) {
    if (!h) return fail(nullptr, IBEM_ERR_ARG, "null handle");
    Plan& P = h->P;
    cudaError_t e;
    if ((e = set_device(h))) return cuda_fail(h, e, "cudaSetDevice");
    if (!h->d_near) {
        size_t nn = (size_t)(P.n_near > 0 ? P.n_near : 1) * P.nb * P.nb * (h->helm ? 2 : 1);
        if ((e = cudaMalloc(&h->d_near, nn * sizeof(double)))) return cuda_fail(h, e, "alloc near blocks");
        if (!h->d_near32 && (e = cudaMalloc(&h->d_near32, nn * sizeof(float))))
            return cuda_fail(h, e, "alloc near blocks fp32");
        if (P.n_far > 0 && h->helm) {
            // stored complex coupling (16 B per entry) if it fits in half of the free memory
            size_t nk = (size_t)P.n_far * h->kpt * 4 * P.q2;
            size_t free_b = 0, total_b = 0;
            cudaMemGetInfo(&free_b, &total_b);
            h->far_on_the_fly = P.prm.fp64_coupling != IBEM_COUPLING_DF || nk * sizeof(float4) > free_b / 2;
            if (P.prm.fp64_coupling == IBEM_COUPLING_FP32_ONLY) h->far_on_the_fly = true;
            if (!h->far_on_the_fly)
                if ((e = cudaMalloc(&h->d_Kc, nk * sizeof(float4)))) return cuda_fail(h, e, "alloc coupling matrices");
        } else if (P.n_far > 0 && P.prm.fp64_coupling != IBEM_COUPLING_NONE &&
                   P.prm.fp64_coupling != IBEM_COUPLING_FP32_ONLY) {   // Laplace (GENERATE: as DF)
            size_t nk = (size_t)P.n_far * h->kpt * 4 * P.q2;
            if (P.prm.fp64_coupling == IBEM_COUPLING_NATIVE) {
                if ((e = cudaMalloc(&h->d_K, nk * sizeof(double)))) return cuda_fail(h, e, "alloc coupling matrices");
            } else {
                size_t nku = (size_t)(h->n_up > 0 ? h->n_up : 1) * h->kpt * 4 * P.q2;
                if ((e = cudaMalloc(&h->d_Kdf, nku * sizeof(float2)))) return cuda_fail(h, e, "alloc coupling matrices");
            }
        }
    }
    if (h->helm) {
        if ((e = helm_launch_near_assembly(h))) return cuda_fail(h, e, "near assembly");
        if ((e = helm_launch_far_assembly(h))) return cuda_fail(h, e, "far assembly");
    } else {
        if ((e = launch_near_assembly(h))) return cuda_fail(h, e, "near assembly");
        if ((e = launch_far_assembly(h))) return cuda_fail(h, e, "far assembly");
    }
    if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(h, e, "assemble sync");
    // work vectors sized before assembly lack the stored coupling's moment buffer
    if (h->d_Kc && !h->d_xh4) h->ws_nrhs = 0;
    if (!h->d_bj_inv) {
        std::string msg;
        if ((e = build_block_jacobi(h, &msg))) return msg.empty() ? cuda_fail(h, e, "block-Jacobi") : fail(h, IBEM_ERR_BREAKDOWN, msg);
    }
    if (!h->helm && h->d_Kdf && !h->up_rows.empty())
        if ((e = tune_coupling_df(h))) return cuda_fail(h, e, "coupling autotune");
    if (P.prm.fp32_coupling == IBEM_FP32_COUPLING_STORE && mr_store_possible(h) && !h->d_Kbf) {
        // if it does not fit, the path keeps generating the coupling
        ibem_status s = store_bf16_coupling(h);
        if (s == IBEM_ERR_OOM) {
            cudaGetLastError();   // a refused allocation is not an error of the assembly
            h->err.clear();
        } else if (s != IBEM_OK) {
            return s;
        }
    }
    if (P.prm.fp64_coupling == IBEM_COUPLING_FP32_ONLY && h->d_near) {
        // the FP32 copy, the diagonal and the block-Jacobi inverses are formed
        if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(h, e, "assemble sync");
        cudaFree(h->d_near);
        h->d_near = nullptr;
    }
    h->assembled = true;
    return IBEM_OK;
}

ibem_status ibem_set_fp32_coupling(ibem_handle* h, int mode) {
    if (!h) return fail(nullptr, IBEM_ERR_ARG, "null handle");
    if (mode != IBEM_FP32_COUPLING_GENERATE && mode != IBEM_FP32_COUPLING_STORE)
        return fail(h, IBEM_ERR_ARG, "mode must be IBEM_FP32_COUPLING_GENERATE or IBEM_FP32_COUPLING_STORE");
    if (!h->assembled) return fail(h, IBEM_ERR_STATE, "ibem_assemble first");
    cudaError_t e;
    if ((e = cudaSetDevice(h->device))) return cuda_fail(h, e, "cudaSetDevice");
    if (mode == IBEM_FP32_COUPLING_GENERATE) {
        if (h->d_Kbf) {
            if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(h, e, "sync");
            cudaFree(h->d_Kbf);
            h->d_Kbf = nullptr;
        }
        h->P.prm.fp32_coupling = mode;
        return IBEM_OK;
    }
    if (!mr_store_possible(h))
        return fail(h, IBEM_ERR_ARG, "stored coupling needs a Helmholtz handle with q_cheb = 8 and far blocks");
    if (!h->d_Kbf) {
        ibem_status s = store_bf16_coupling(h);
        if (s != IBEM_OK) return s;
    }
    h->P.prm.fp32_coupling = mode;
    return IBEM_OK;
}

ibem_status ibem_quad_points(const ibem_handle* hc, double* xyz_dev) {
    ibem_handle* h = const_cast<ibem_handle*>(hc);
    if (!h || !xyz_dev) return fail(h, IBEM_ERR_ARG, "null handle or output");
    cudaError_t e = cudaMemcpy2DAsync(xyz_dev, 3 * sizeof(double), h->d_qgeo, 4 * sizeof(double), 3 * sizeof(double),
                                      (size_t)h->P.nq, cudaMemcpyDeviceToDevice, h->stream);
    if (e) return cuda_fail(h, e, "quad points copy");
    return IBEM_OK;
}

ibem_status ibem_rhs(ibem_handle* h, const double* g_dev, int nrhs, double* b_dev) {
    if (!h) return fail(nullptr, IBEM_ERR_ARG, "null handle");
    if (nrhs < 0 || (nrhs > 0 && (!g_dev || !b_dev))) return fail(h, IBEM_ERR_ARG, "bad rhs arguments");
    if (nrhs == 0) return IBEM_OK;
    cudaError_t e;
    if ((e = set_device(h))) return cuda_fail(h, e, "cudaSetDevice");
    if ((e = launch_rhs(h, g_dev, nrhs, b_dev))) return cuda_fail(h, e, "rhs");
    return IBEM_OK;
}

ibem_status ibem_matvec(ibem_handle* h, const double* x_dev, double* y_dev, int nrhs, int precision) {
    ibem_status s = check_ready(h);
    if (s) return s;
    if (nrhs < 0 || (nrhs > 0 && (!x_dev || !y_dev))) return fail(h, IBEM_ERR_ARG, "bad matvec arguments");
    if (precision != IBEM_FP64 && precision != IBEM_FP32) return fail(h, IBEM_ERR_ARG, "unknown precision");
    if (x_dev == y_dev) return fail(h, IBEM_ERR_ARG, "x and y must not overlap");
    if (nrhs == 0) return IBEM_OK;
    if (precision == IBEM_FP64 && !fp64_available(h))
        return fail(h, IBEM_ERR_STATE, "no FP64 coupling stored (IBEM_COUPLING_NONE)");
    cudaError_t e;
    if ((e = set_device(h))) return cuda_fail(h, e, "cudaSetDevice");
    if ((e = apply_operator(h, x_dev, y_dev, nrhs, precision))) return cuda_fail(h, e, "matvec");
    return IBEM_OK;
}

ibem_status ibem_matvec_host(ibem_handle* h, const double* x, double* y, int nrhs, int precision) {
    ibem_status s = check_ready(h);
    if (s) return s;
    if (precision == IBEM_FP64 && !fp64_available(h))
        return fail(h, IBEM_ERR_STATE, "no FP64 coupling stored (IBEM_COUPLING_NONE)");
    if (nrhs < 0 || (nrhs > 0 && (!x || !y))) return fail(h, IBEM_ERR_ARG, "bad matvec arguments");
    if (nrhs == 0) return IBEM_OK;
    cudaError_t e;
    if ((e = set_device(h))) return cuda_fail(h, e, "cudaSetDevice");
    // [nrhs][ndof] values, complex (two doubles each) for Helmholtz
    size_t bytes = (size_t)nrhs * h->P.N * (h->helm ? 2 : 1) * sizeof(double);
    double *dx = nullptr, *dy = nullptr;
    if ((e = cudaMallocAsync(&dx, bytes, h->stream))) return cuda_fail(h, e, "alloc x");
    if ((e = cudaMallocAsync(&dy, bytes, h->stream))) { cudaFreeAsync(dx, h->stream); return cuda_fail(h, e, "alloc y"); }
    e = cudaMemcpyAsync(dx, x, bytes, cudaMemcpyHostToDevice, h->stream);
    if (!e) e = apply_operator(h, dx, dy, nrhs, precision);
    if (!e) e = cudaMemcpyAsync(y, dy, bytes, cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(dx, h->stream);
    cudaFreeAsync(dy, h->stream);
    cudaError_t e2 = cudaStreamSynchronize(h->stream);
    if (e) return cuda_fail(h, e, "matvec_host");
    if (e2) return cuda_fail(h, e2, "matvec_host sync");
    return IBEM_OK;
}

ibem_status ibem_solve(ibem_handle* h, const double* b_dev, double* w_dev, int nrhs, double rtol, int maxit,
                       int precond, int precision, ibem_solve_info* info) {
    ibem_status s = check_ready(h);
    if (s) return s;
    if (nrhs < 0 || (nrhs > 0 && (!b_dev || !w_dev)) || !(rtol > 0.0) || maxit < 1)
        return fail(h, IBEM_ERR_ARG, "bad solve arguments");
    if (precond != IBEM_PRECOND_NONE && precond != IBEM_PRECOND_JACOBI && precond != IBEM_PRECOND_BLOCK_JACOBI &&
        precond != IBEM_PRECOND_LEARNED)
        return fail(h, IBEM_ERR_ARG, "unknown preconditioner");
    if (precond == IBEM_PRECOND_LEARNED && (!h->helm || !h->cnn))
        return fail(h, IBEM_ERR_STATE, "learned preconditioner: Helmholtz handle with an attached network required");
    if (precision != IBEM_FP64 && precision != IBEM_FP32) return fail(h, IBEM_ERR_ARG, "unknown precision");
    if (nrhs == 0) return IBEM_OK;
    if (!fp64_available(h)) return fail(h, IBEM_ERR_STATE, "no FP64 coupling stored (IBEM_COUPLING_NONE)");
    cudaError_t e;
    if ((e = set_device(h))) return cuda_fail(h, e, "cudaSetDevice");
    s = solve_impl(h, b_dev, w_dev, nrhs, rtol, maxit, precond, precision, info);
    if (s == IBEM_ERR_NOCONV) h->err = "solver did not reach rtol within maxit";
    else if (s == IBEM_ERR_BREAKDOWN) h->err = "solver breakdown";
    else if (s != IBEM_OK) h->err = "solver failed (CUDA error)";
    return s;
}

ibem_status ibem_set_learned_preconditioner(ibem_handle* h, ibem_cnn* cnn) {
    if (!h) return fail(nullptr, IBEM_ERR_ARG, "null handle");
    if (cnn && !h->helm) return fail(h, IBEM_ERR_ARG, "the learned preconditioner is for Helmholtz handles");
    h->cnn = cnn;
    return IBEM_OK;
}

ibem_status ibem_learned_apply(ibem_handle* h, const double* v_dev, double* z_dev) {
    ibem_status s = check_ready(h);
    if (s) return s;
    if (!v_dev || !z_dev || v_dev == z_dev) return fail(h, IBEM_ERR_ARG, "bad learned_apply arguments");
    if (!h->helm || !h->cnn) return fail(h, IBEM_ERR_STATE, "no learned preconditioner attached");
    cudaError_t e;
    if ((e = set_device(h))) return cuda_fail(h, e, "cudaSetDevice");
    if ((e = cnn_precondition(h, h->cnn, v_dev, z_dev))) return cuda_fail(h, e, "learned preconditioner");
    return IBEM_OK;
}

ibem_status ibem_solver_pairs(ibem_handle* h, const double* b_dev, int nrhs, double rtol, int maxit, int stride,
                              int max_pairs, float* in_img_dev, float* tgt_img_dev, int* n_pairs,
                              ibem_solve_info* info) {
    ibem_status s = check_ready(h);
    if (s) return s;
    if (!h->helm) return fail(h, IBEM_ERR_ARG, "solver pairs are generated for Helmholtz handles");
    if (nrhs < 1 || !b_dev || !in_img_dev || !tgt_img_dev || !n_pairs || !(rtol > 0.0) || maxit < 1 || stride < 1 ||
        max_pairs < 1)
        return fail(h, IBEM_ERR_ARG, "bad solver_pairs arguments");
    if (!fp64_available(h)) return fail(h, IBEM_ERR_STATE, "no FP64 coupling stored (IBEM_COUPLING_NONE)");
    cudaError_t e;
    if ((e = set_device(h))) return cuda_fail(h, e, "cudaSetDevice");
    *n_pairs = 0;
    s = solver_pairs_impl(h, b_dev, nrhs, rtol, maxit, stride, max_pairs, in_img_dev, tgt_img_dev, n_pairs, info);
    if (s == IBEM_ERR_NOCONV) h->err = "a solve of the pair generation did not reach rtol (pairs kept)";
    else if (s != IBEM_OK) h->err = "pair generation failed";
    return s;
}

ibem_status ibem_solver_residuals(ibem_handle* h, const double* b_dev, int nrhs, double rtol, int maxit, int stride,
                                  int max_vecs, double* r_out_dev, int* n_out, ibem_solve_info* info) {
    ibem_status s = check_ready(h);
    if (s) return s;
    if (!h->helm) return fail(h, IBEM_ERR_ARG, "solver residuals are generated for Helmholtz handles");
    if (nrhs < 1 || !b_dev || !r_out_dev || !n_out || !(rtol > 0.0) || maxit < 1 || stride < 1 || max_vecs < 1)
        return fail(h, IBEM_ERR_ARG, "bad solver_residuals arguments");
    if (!fp64_available(h)) return fail(h, IBEM_ERR_STATE, "no FP64 coupling stored (IBEM_COUPLING_NONE)");
    cudaError_t e;
    if ((e = set_device(h))) return cuda_fail(h, e, "cudaSetDevice");
    *n_out = 0;
    s = solver_residuals_impl(h, b_dev, nrhs, rtol, maxit, stride, max_vecs, r_out_dev, n_out, info);
    if (s == IBEM_ERR_NOCONV) h->err = "a solve of the residual generation did not reach rtol (vectors kept)";
    else if (s != IBEM_OK) h->err = "residual generation failed";
    return s;
}

ibem_status ibem_profile_enable(ibem_handle* h, int enable) {
    if (!h) return fail(nullptr, IBEM_ERR_ARG, "null handle");
    ibem_profile_data scratch;
    ibem_status s = ibem_profile_read(h, &scratch);
    if (s) return s;
    h->prof = enable != 0;
    return IBEM_OK;
}

ibem_status ibem_profile_read(ibem_handle* h, ibem_profile_data* out) {
    if (!h || !out) return fail(nullptr, IBEM_ERR_ARG, "null handle or output");
    cudaError_t e;
    if ((e = set_device(h))) return cuda_fail(h, e, "cudaSetDevice");
    if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(h, e, "profile sync");
    std::memset(out, 0, sizeof(*out));
    for (auto& u : h->ev_used) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, u.second.first, u.second.second) == cudaSuccess && u.first >= 0 && u.first < 6)
            out->ms[u.first] += ms;
        h->ev_free.push_back(u.second.first);
        h->ev_free.push_back(u.second.second);
    }
    h->ev_used.clear();
    out->applications = h->applications;
    out->launches = h->launches;
    h->applications = 0;
    h->launches = 0;
    return IBEM_OK;
}

ibem_status ibem_set_wait_limit(ibem_handle* h, long long limit) {
    if (!h || limit < 0) return fail(h, IBEM_ERR_ARG, "null handle or negative limit");
    h->wait_limit = limit;
    return IBEM_OK;
}

ibem_status ibem_device_status(ibem_handle* h, int* status) {
    if (!h || !status) return fail(h, IBEM_ERR_ARG, "null handle or output");
    cudaError_t e;
    if ((e = set_device(h))) return cuda_fail(h, e, "cudaSetDevice");
    if ((e = cudaMemcpyAsync(status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream)))
        return cuda_fail(h, e, "status read");
    if ((e = cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream))) return cuda_fail(h, e, "status clear");
    if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(h, e, "status sync");
    return IBEM_OK;
}

ibem_status ibem_potential(ibem_handle* h, const double* w_dev, int nrhs, const double* pts_dev, int64_t npts,
                           double* u_dev) {
    if (!h) return fail(nullptr, IBEM_ERR_ARG, "null handle");
    if (nrhs < 0 || npts < 0 || (nrhs > 0 && npts > 0 && (!w_dev || !pts_dev || !u_dev)))
        return fail(h, IBEM_ERR_ARG, "bad potential arguments");
    if (nrhs == 0 || npts == 0) return IBEM_OK;
    cudaError_t e;
    if ((e = set_device(h))) return cuda_fail(h, e, "cudaSetDevice");
    if ((e = launch_potential(h, w_dev, nrhs, pts_dev, npts, u_dev))) return cuda_fail(h, e, "potential");
    return IBEM_OK;
}

ibem_status ibem_potential_fmm(ibem_handle* h, const double* w_dev, int nrhs, const double* pts_dev, int64_t npts,
                               double* u_dev, int64_t* n_far_terms, int64_t* n_near_terms) {
    if (!h) return fail(nullptr, IBEM_ERR_ARG, "null handle");
    if (nrhs < 0 || npts < 0 || (nrhs > 0 && npts > 0 && (!w_dev || !pts_dev || !u_dev)))
        return fail(h, IBEM_ERR_ARG, "bad potential arguments");
    if (h->P.q == 0) return fail(h, IBEM_ERR_ARG, "ibem_potential_fmm needs a compressed handle (q_cheb > 0)");
    if (npts > 2147483647LL || nrhs > 262140)   // grid.x = points; grid.y of the moments = 2 nrhs / 8 <= 65535
        return fail(h, IBEM_ERR_ARG, "ibem_potential_fmm takes at most 2^31 - 1 points and 262,140 densities");
    if (n_far_terms) *n_far_terms = 0;
    if (n_near_terms) *n_near_terms = 0;
    if (nrhs == 0 || npts == 0) return IBEM_OK;
    cudaError_t e;
    if ((e = set_device(h))) return cuda_fail(h, e, "cudaSetDevice");
    if ((e = launch_potential_fmm(h, w_dev, nrhs, pts_dev, npts, u_dev, n_far_terms, n_near_terms)))
        return cuda_fail(h, e, "potential_fmm");
    return IBEM_OK;
}

ibem_status ibem_rhs_sources(ibem_handle* h, const double* src_dev, const double* charges_dev, int nrhs,
                             int64_t nsrc, double* b_dev, int64_t* n_far_terms, int64_t* n_near_terms) {
    if (!h) return fail(nullptr, IBEM_ERR_ARG, "null handle");
    if (nrhs < 0 || nsrc < 0 || (nrhs > 0 && !b_dev) || (nrhs > 0 && nsrc > 0 && (!src_dev || !charges_dev)))
        return fail(h, IBEM_ERR_ARG, "bad right-hand-side arguments");
    if (h->P.q == 0) return fail(h, IBEM_ERR_ARG, "ibem_rhs_sources needs a compressed handle (q_cheb > 0)");
    if (nsrc > 2147483647LL || nrhs > 32767)   // grid.x = sources; grid.y of the downward pass = 2 nrhs
        return fail(h, IBEM_ERR_ARG, "ibem_rhs_sources takes at most 2^31 - 1 sources and 32,767 charge vectors");
    if (n_far_terms) *n_far_terms = 0;
    if (n_near_terms) *n_near_terms = 0;
    if (nrhs == 0) return IBEM_OK;
    cudaError_t e;
    if ((e = set_device(h))) return cuda_fail(h, e, "cudaSetDevice");
    if (nsrc == 0) {
        const size_t n = (size_t)nrhs * h->P.N * (h->helm ? 2 : 1);
        if ((e = cudaMemsetAsync(b_dev, 0, n * sizeof(double), h->stream))) return cuda_fail(h, e, "memset");
        return IBEM_OK;
    }
    if ((e = launch_rhs_sources(h, src_dev, charges_dev, nrhs, nsrc, b_dev, n_far_terms, n_near_terms)))
        return cuda_fail(h, e, "rhs_sources");
    return IBEM_OK;
}

}  // extern "C"
