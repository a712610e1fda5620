// Internal declarations of libibem: patch evaluation (host + device), the
// handle, launch helpers.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ibem.h"

#define IBEM_MAX_DEG 7      // NURBS degree limit
#define IBEM_MAX_P 4        // spline degree limit
#define IBEM_MAX_NB 25      // (IBEM_MAX_P + 1)^2 Bernstein functions per element
#define IBEM_MAX_GAUSS 40   // Gauss points per direction of the regular rule
#define IBEM_MAX_SMEM_BYTES 232448   // dynamic shared memory one CTA may use (227 KB)
#define IBEM_MAX_Q 12       // Chebyshev points per direction
#define IBEM_PI 3.14159265358979323846

namespace ibem {

// ---------------------------------------------------------------------------
// Patch description usable on host and device (Sec. 2.2, Eq. def::geom).
// ---------------------------------------------------------------------------
struct PatchDesc {
    int kind;                 // IBEM_PATCH_*
    int deg_u, deg_v, ncp_u, ncp_v;
    int knot_off_u, knot_off_v, cp_off;   // offsets into knots[] and cpw[] (x w, y w, z w, w)
    double R, c0[3], n[3], t1[3], t2[3];  // sphere face
    int perturbed;            // parameters mapped by perturbation_f first
};

struct GeomView {
    const PatchDesc* patches;
    const double* knots;
    const double* cpw;
};

// Index of the knot span [xi_s, xi_{s+1}) containing u for a p-open knot vector
// with ncp control points; u = 1 belongs to the last non-empty span.
__host__ __device__ inline int find_span(const double* xi, int deg, int ncp, double u) {
    int s = deg;
    for (int j = deg; j < ncp; ++j)
        if (xi[j] <= u && xi[j] < xi[j + 1]) s = j;
    return s;
}

// Non-zero B-splines b_{s-deg..s} of degree deg at u and their derivatives,
// by the Cox-de Boor recursion (Def. 2.1) on the local triangle.
__host__ __device__ inline void local_bsplines(const double* xi, int deg, int s, double u,
                                               double* val, double* der) {
    double b[IBEM_MAX_DEG + 2];
    for (int k = 0; k <= deg + 1; ++k) b[k] = 0.0;
    b[deg] = 1.0;                                   // degree 0: only b_s is non-zero
    double lower[IBEM_MAX_DEG + 2];
    for (int d = 1; d <= deg; ++d) {
        if (d == deg)
            for (int k = 0; k <= deg + 1; ++k) lower[k] = b[k];
        double nb[IBEM_MAX_DEG + 2];
        for (int k = 0; k <= deg; ++k) {
            int j = s - deg + k;
            double t = 0.0;
            double den1 = xi[j + d] - xi[j];
            double den2 = xi[j + d + 1] - xi[j + 1];
            if (den1 > 0.0) t += (u - xi[j]) / den1 * b[k];
            if (den2 > 0.0) t += (xi[j + d + 1] - u) / den2 * b[k + 1];
            nb[k] = t;
        }
        nb[deg + 1] = 0.0;
        for (int k = 0; k <= deg + 1; ++k) b[k] = nb[k];
    }
    if (deg == 0) {
        for (int k = 0; k <= deg; ++k) { val[k] = b[k]; der[k] = 0.0; }
        return;
    }
    for (int k = 0; k <= deg; ++k) {
        int j = s - deg + k;
        double dd = 0.0;
        double den1 = xi[j + deg] - xi[j];
        double den2 = xi[j + deg + 1] - xi[j + 1];
        if (den1 > 0.0) dd += deg / den1 * lower[k];
        if (den2 > 0.0) dd -= deg / den2 * lower[k + 1];
        val[k] = b[k];
        der[k] = dd;
    }
}

// The piecewise-linear reparametrisation of [0, 1] of Sec. 5 (perturbed
// mappings): slopes 1/2, 7/4, 1/2 with kinks at 0.3 and 0.7; returns f(x) and
// stores f'(x) (the left piece's slope at a kink, which no quadrature or
// interpolation point of a dyadic mesh hits).
__host__ __device__ inline double perturbation_f(double x, double* df) {
    if (x <= 0.3) { *df = 0.5; return 0.5 * x; }
    if (x < 0.7) { *df = 1.75; return 1.75 * x - 0.375; }
    *df = 0.5;
    return 0.5 * (x + 1.0);
}

__host__ __device__ inline void eval_patch_map(const PatchDesc& P, const GeomView& g, double u, double v,
                                               double F[3], double Fu[3], double Fv[3]);

// F(u, v), dF/du, dF/dv of one patch (chain rule through f for a perturbed patch).
__host__ __device__ inline void eval_patch(const GeomView& g, int ip, double u, double v,
                                           double F[3], double Fu[3], double Fv[3]) {
    const PatchDesc& P = g.patches[ip];
    if (P.perturbed) {
        double du, dv;
        const double fu = perturbation_f(u, &du), fv = perturbation_f(v, &dv);
        eval_patch_map(P, g, fu, fv, F, Fu, Fv);
        for (int i = 0; i < 3; ++i) {
            Fu[i] *= du;
            Fv[i] *= dv;
        }
        return;
    }
    eval_patch_map(P, g, u, v, F, Fu, Fv);
}

// The patch map itself: analytic sphere face or NURBS.
__host__ __device__ inline void eval_patch_map(const PatchDesc& P, const GeomView& g, double u, double v,
                                               double F[3], double Fu[3], double Fv[3]) {
    if (P.kind == IBEM_PATCH_SPHERE_FACE) {
        double a = 2.0 * u - 1.0, b = 2.0 * v - 1.0;
        double c[3];
        for (int i = 0; i < 3; ++i) c[i] = P.n[i] + a * P.t1[i] + b * P.t2[i];
        double r2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        double r = sqrt(r2);
        double ct1 = c[0] * P.t1[0] + c[1] * P.t1[1] + c[2] * P.t1[2];
        double ct2 = c[0] * P.t2[0] + c[1] * P.t2[1] + c[2] * P.t2[2];
        for (int i = 0; i < 3; ++i) {
            F[i] = P.c0[i] + (P.R * c[i]) / r;
            Fu[i] = P.R * 2.0 * (P.t1[i] - c[i] * (ct1 / r2)) / r;
            Fv[i] = P.R * 2.0 * (P.t2[i] - c[i] * (ct2 / r2)) / r;
        }
        return;
    }
    const double* xu = g.knots + P.knot_off_u;
    const double* xv = g.knots + P.knot_off_v;
    int su = find_span(xu, P.deg_u, P.ncp_u, u);
    int sv = find_span(xv, P.deg_v, P.ncp_v, v);
    double bu[IBEM_MAX_DEG + 1], du[IBEM_MAX_DEG + 1], bv[IBEM_MAX_DEG + 1], dv[IBEM_MAX_DEG + 1];
    local_bsplines(xu, P.deg_u, su, u, bu, du);
    local_bsplines(xv, P.deg_v, sv, v, bv, dv);
    double S[4] = {0, 0, 0, 0}, Su[4] = {0, 0, 0, 0}, Sv[4] = {0, 0, 0, 0};
    for (int kv = 0; kv <= P.deg_v; ++kv) {
        int jv = sv - P.deg_v + kv;
        for (int ku = 0; ku <= P.deg_u; ++ku) {
            int ju = su - P.deg_u + ku;
            const double* cp = g.cpw + P.cp_off + 4 * (jv * P.ncp_u + ju);
            double w0 = bu[ku] * bv[kv], wu = du[ku] * bv[kv], wv = bu[ku] * dv[kv];
            for (int i = 0; i < 4; ++i) {
                S[i] += w0 * cp[i];
                Su[i] += wu * cp[i];
                Sv[i] += wv * cp[i];
            }
        }
    }
    for (int i = 0; i < 3; ++i) {
        F[i] = S[i] / S[3];
        Fu[i] = (Su[i] - F[i] * Su[3]) / S[3];
        Fv[i] = (Sv[i] - F[i] * Sv[3]) / S[3];
    }
}

__host__ __device__ inline double surface_measure(const double Fu[3], const double Fv[3]) {
    double n0 = Fu[1] * Fv[2] - Fu[2] * Fv[1];
    double n1 = Fu[2] * Fv[0] - Fu[0] * Fv[2];
    double n2 = Fu[0] * Fv[1] - Fu[1] * Fv[0];
    return sqrt(n0 * n0 + n1 * n1 + n2 * n2);
}

// Bernstein polynomials B_{i,p}(t) = C(p,i) t^i (1-t)^{p-i}, i = 0..p (Sec. 4.3).
__host__ __device__ inline void bernstein(int p, double t, double* out) {
    double s = 1.0 - t;
    // de Casteljau-style build-up: degree d from degree d-1
    out[0] = 1.0;
    for (int d = 1; d <= p; ++d) {
        double prev = 0.0;
        for (int i = 0; i < d; ++i) {
            double cur = out[i];
            out[i] = prev + s * cur;
            prev = t * cur;
        }
        out[d] = prev;
    }
}

// Morton (Z-order) interleave of (x, y), x in the even bits (16-bit inputs).
__host__ __device__ inline uint32_t spread_bits(uint32_t v) {
    v &= 0x0000FFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
__host__ __device__ inline uint32_t compact_bits(uint32_t v) {
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0F0F0F0Fu;
    v = (v | (v >> 4)) & 0x00FF00FFu;
    v = (v | (v >> 8)) & 0x0000FFFFu;
    return v;
}
__host__ __device__ inline uint32_t morton2(uint32_t x, uint32_t y) { return spread_bits(x) | (spread_bits(y) << 1); }
__host__ __device__ inline void morton2_inv(uint32_t z, uint32_t* x, uint32_t* y) {
    *x = compact_bits(z);
    *y = compact_bits(z >> 1);
}

// The eight symmetries rho_k(s,t) = (a0 + a1 s + a2 t, b0 + b1 s + b2 t) of the
// unit square in a fixed order (identity, rotations by 90/180/270 degrees, the
// four reflections).  The order decides which canonical orientation a touching
// pair gets, so it is part of the quadrature rule.
__host__ __device__ inline void dihedral(int k, double s, double t, double* x, double* y) {
    switch (k) {
        case 0: *x = s; *y = t; break;
        case 1: *x = 1.0 - t; *y = s; break;
        case 2: *x = 1.0 - s; *y = 1.0 - t; break;
        case 3: *x = t; *y = 1.0 - s; break;
        case 4: *x = t; *y = s; break;
        case 5: *x = 1.0 - s; *y = t; break;
        case 6: *x = 1.0 - t; *y = 1.0 - s; break;
        default: *x = s; *y = 1.0 - t; break;
    }
}

enum PairClass { CLS_IDENTICAL = 0, CLS_EDGE = 1, CLS_VERTEX = 2, CLS_SUBDIV = 3, CLS_REGULAR = 4 };

// ---------------------------------------------------------------------------
// Host-side discretisation and tree (setup.cu)
// ---------------------------------------------------------------------------
struct Plan {
    ibem_params prm;
    int npatch = 0, p = 0, m = 0, pp = 1, nb = 1, ne1 = 1, n1 = 1, Q = 8, Qs = 8, q = 0, q2 = 0;
    int64_t E = 0, N = 0, Nstar = 0, C = 0, nq = 0;
    std::vector<PatchDesc> patches;
    std::vector<double> knots, cpw;
    GeomView host_view() const { return GeomView{patches.data(), knots.data(), cpw.data()}; }
    // element e = patch * 4^m + morton(ix, iy); cluster id = level_off[l] + patch * 4^l + morton
    std::vector<int64_t> level_off;
    // near field: CSR by target element (sources ascending)
    std::vector<int64_t> near_ptr;
    std::vector<int32_t> near_src, near_cls, near_orient;
    std::vector<int32_t> near_order;   // Gauss order per direction of every near pair
    int max_order = 0;                 // largest order of a non-touching near pair
    int64_t n_graded = 0;              // non-touching pairs with order != Q
    // far field: CSR by target cluster id (sources ascending)
    std::vector<int64_t> far_ptr;
    std::vector<int32_t> far_src;
    int64_t n_near = 0, n_far = 0, n_cls[5] = {0, 0, 0, 0, 0};
    // bounding ball of every cluster, [C][4] = (centre x, y, z, radius)
    std::vector<double> balls;
};

std::string build_plan(const ibem_patch* patches, int npatch, const ibem_params* prm, Plan& P);
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
void chebyshev_nodes(int q, std::vector<double>& z);
void lagrange_values(const std::vector<double>& z, double x, double* L);
void element_of(const Plan& P, int64_t e, int* patch, int* ix, int* iy);
void cluster_of(const Plan& P, int64_t c, int* patch, int* level, int* ix, int* iy);
// Canonical rules (x1, x2, y1, y2, w) of the touching classes, SoA [5][n].
void singular_rule(int cls, int n, std::vector<double>& soa);

}  // namespace ibem

// ---------------------------------------------------------------------------
// The handle
// ---------------------------------------------------------------------------
struct ibem_cnn;

struct ibem_handle {
    ibem::Plan P;
    cudaStream_t stream = nullptr;
    int device = 0;
    bool helm = false;
    bool assembled = false;
    std::string err;

    // geometry and tables
    ibem::PatchDesc* d_patches = nullptr;
    double* d_knots = nullptr;
    double* d_cpw = nullptr;
    double* d_ext = nullptr;        // Bezier extraction [ne1][pp][pp]: b_{ix+r} = sum_i ext[ix][r][i] B_i
    double* d_qgeo = nullptr;       // [E][Q*Q][4] = (x, y, z, gauss weight * k * h^2)
    double* d_igeo = nullptr;       // [C][q2][4]  = (x, y, z, k) at interpolation points
    double* d_balls = nullptr;      // [C][4] cluster bounding balls (centre, radius)
    double* d_mu1d = nullptr;       // 1D cluster moment tables of every level (interpolated potential)
    int64_t* d_mu1d_off = nullptr;  // their offsets per level
    float* d_igeo32 = nullptr;      // same in FP32
    double* d_phi = nullptr;        // [Q*Q][nb] Bernstein products at the regular Gauss points
    double* d_phi_sub = nullptr;    // [4][Q*Q][nb] at the 2x2-subdivided Gauss points
    double* d_rule[3] = {nullptr, nullptr, nullptr};  // singular rules, SoA [5][n]
    int rule_n[3] = {0, 0, 0};
    double* d_M = nullptr;          // [q][pp] 1D leaf moments int L_a B_i (times h)
    double* d_S = nullptr;          // [2][q][q] 1D M2M: S_c[a][b] = L_a((c + z_b) / 2)
    float* d_Mf = nullptr;          // FP32 copies of M and S for the FP32 many-right-hand-side path
    float* d_Sf = nullptr;

    // near field
    int64_t* d_near_ptr = nullptr;
    int32_t* d_near_src = nullptr;
    int32_t* d_near_tgt = nullptr;
    int32_t* d_near_cls = nullptr;
    int32_t* d_near_orient = nullptr;
    int32_t* d_pairs_by_cls[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int64_t n_list[5] = {0, 0, 0, 0, 0};   // lengths of d_pairs_by_cls (graded pairs excluded)
    // graded near pairs (order != Q): one group per (class, order), its pairs
    // contiguous in d_graded_pairs, its rule (nodes, weights) and Bernstein
    // table ([1 or 4][n^2][nb]) at tab_off in d_graded_tab
    struct GradedGroup {
        int cls, order;
        int64_t off, count;
        size_t tab_off;
    };
    std::vector<GradedGroup> graded;
    int32_t* d_graded_pairs = nullptr;
    double* d_graded_tab = nullptr;
    double* d_near = nullptr;       // [n_near][nb][nb] (complex: [..][2])
    float* d_near32 = nullptr;

    // far field
    int64_t* d_far_ptr = nullptr;
    int32_t* d_far_src = nullptr;
    int32_t* d_far_tgt = nullptr;
    double* d_K = nullptr;          // [n_far][kpt][4 q2]: entry (a, b = s + 4k) at [k][4a + s] (native)
    float2* d_Kdf = nullptr;        // same layout, (hi, lo) float pairs (double-float coupling)
    float2* d_xh2 = nullptr;        // forward moments split into (hi, lo) float pairs
    float4* d_Kc = nullptr;         // Helmholtz: double-float complex coupling (re_hi, re_lo, im_hi, im_lo)
    float4* d_xh4 = nullptr;        // Helmholtz: forward moments as double-float complex
    double* d_hsx = nullptr;        // Helmholtz: split-layout input  [2R][max(N, nq)]
    double* d_hsy = nullptr;        // Helmholtz: split-layout output [2R][N]
    bool far_on_the_fly = false;    // Helmholtz FP64 coupling generated on the fly (stored K too large)
    double far_diam = 0.0;          // bound on the distance of two points of a far block (cluster balls)
    float4* d_gen_pts = nullptr;    // double-float point tables [C][q2][2] of the generated coupling
    float4* d_gen_trig = nullptr;   // e^{i j 2 pi / 2048} as double-float pairs
    float4* d_gen_x = nullptr;      // moments, chunked double-float complex [nch][C][q2][RC]
    size_t gen_x_bytes = 0;
    int kpt = 0;
    int df_nst = 0;   // ring depth of the double-float coupling (autotuned at assembly; 0 = default)
    std::vector<int32_t> far_rows;  // target clusters with a non-empty far list
    int max_far_row = 0;            // longest far list
    // upper half of the far field (source id > target id), used with symmetric storage
    std::vector<int32_t> up_rows;
    int max_up_row = 0;
    int64_t n_up = 0;
    int64_t* d_up_ptr = nullptr;
    int32_t* d_up_src = nullptr;
    int32_t* d_up_tgt = nullptr;
    int32_t* d_up_rows = nullptr;
    int64_t* d_tr_ptr = nullptr;    // transposed upper list: for each source cluster, its stored blocks
    int32_t* d_tr_blk = nullptr;
    float2* d_colpart = nullptr;    // per stored block and right-hand side: column share K^T x^_sigma (hi, lo)
    int32_t* d_far_rows = nullptr;

    // work vectors (sized for ws_nrhs right-hand sides)
    int ws_nrhs = 0;
    double *d_xs = nullptr, *d_ys = nullptr, *d_xh = nullptr, *d_yh = nullptr;
    float *d_xs32 = nullptr, *d_ys32 = nullptr, *d_yh32 = nullptr;
    float4* d_src32 = nullptr;
    double* d_diag = nullptr;       // Jacobi diagonal of T A_near T^T
    double* d_solver = nullptr;     // solver work space
    size_t solver_len = 0;
    double* d_red = nullptr;        // reduction scratch
    double* h_red = nullptr;        // pinned host copy of reductions

    // tracing: event pairs per phase while enabled, launch counter always
    bool prof = false;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
    int64_t launches = 0, applications = 0;

    // many-right-hand-side FP32 path (tensor-core coupling): one work area
    void* d_mr = nullptr;
    size_t mr_bytes = 0;
    void* d_Kbf = nullptr;          // stored BF16 coupling blocks [n_far][128][64] (IBEM_FP32_COUPLING_STORE)
    int st_nst = 0;                 // ring depth of the stored-coupling kernel (0: not timed yet)
    void* d_sl = nullptr;           // digit slices and column exponents of the moments (IBEM_COUPLING_SLICED)
    size_t sl_bytes = 0;

    // block-Jacobi preconditioner: blocks of dofs, inverse blocks
    int64_t* d_bj_ptr = nullptr;
    int64_t* d_bj_off = nullptr;
    int32_t* d_bj_dofs = nullptr;
    double* d_bj_inv = nullptr;
    int64_t bj_blocks = 0;

    // learned preconditioner (not owned; IBEM_PRECOND_LEARNED)
    ibem_cnn* cnn = nullptr;

    // device-side waits: bound (polls) and status word (IBEM_DEVICE_* bits)
    long long wait_limit = 1LL << 26;
    int* d_status = nullptr;
};

namespace ibem {
// Phase timer: records an event pair on the stream while profiling is on.
struct PhaseTimer {
    ibem_handle* h;
    int phase;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEvent_t take() {
        cudaEvent_t ev = nullptr;
        if (!h->ev_free.empty()) { ev = h->ev_free.back(); h->ev_free.pop_back(); }
        else cudaEventCreate(&ev);
        return ev;
    }
    PhaseTimer(ibem_handle* hh, int ph) : h(hh), phase(ph) {
        if (!h->prof) return;
        a = take();
        b = take();
        cudaEventRecord(a, h->stream);
    }
    // end the phase now (the destructor then does nothing)
    void stop() {
        if (!a) return;
        cudaEventRecord(b, h->stream);
        h->ev_used.push_back({phase, {a, b}});
        a = nullptr;
    }
    ~PhaseTimer() { stop(); }
};

// real kernels of kernels_apply.cu reused by the complex (Helmholtz) path
__global__ void lift_kernel(int R, int64_t E, int p, int ne1, const double* __restrict__ ext,
                            const double* __restrict__ x, int64_t N, double* __restrict__ xs);
__global__ void restrict_kernel(int R, int64_t N, int p, int ne1, const double* __restrict__ ext,
                                const double* __restrict__ ys, int64_t E, double* __restrict__ y);
__global__ void leaf_moment_kernel(int R, int64_t E, int pp, int q, const double* __restrict__ M,
                                   const double* __restrict__ xs, int64_t leaf_off, int64_t C, double* __restrict__ xh);
__global__ void m2m_kernel(int R, int64_t nL, int64_t offL, int64_t offL1, int q, const double* __restrict__ S,
                           int64_t C, double* __restrict__ xh);
__global__ void l2l_kernel(int R, int64_t nL1, int64_t offL, int64_t offL1, int q, const double* __restrict__ S,
                           int64_t C, double* __restrict__ yh);
__global__ void leaf_back_kernel(int R, int64_t E, int pp, int q, const double* __restrict__ M,
                                 const double* __restrict__ yh, int64_t leaf_off, int64_t C, double* __restrict__ ys);
__global__ void m2m_sep_kernel(int64_t nL, int64_t offL, int64_t offL1, int q, const double* __restrict__ S,
                               int64_t C, double* __restrict__ xh);
__global__ void l2l_sep_kernel(int64_t nL, int64_t offL, int64_t offL1, int q, const double* __restrict__ S,
                               int64_t C, double* __restrict__ yh);
__global__ void d2f_kernel(const double* __restrict__ in, float* __restrict__ out, int64_t n);
__global__ void rhs_super_kernel(int R, int64_t E, int QQ, int nb, const double* __restrict__ qgeo,
                                 const double* __restrict__ phi, const double* __restrict__ g, int64_t nq,
                                 double* __restrict__ gs);
// Helmholtz (kernels_helm.cu)
cudaError_t helm_launch_near_assembly(ibem_handle* h);
cudaError_t helm_launch_far_assembly(ibem_handle* h);
cudaError_t helm_apply_operator(ibem_handle* h, const double* x, double* y, int nrhs, int precision, double* xsplit,
                                double* ysplit);
cudaError_t helm_launch_rhs(ibem_handle* h, const double* g, int nrhs, double* b, double* gsplit, double* bsplit);
cudaError_t helm_launch_potential(ibem_handle* h, const double* w, int nrhs, const double* pts, int64_t npts,
                                  double* u, double* wsplit);
__global__ void helm_split_vec_kernel(int R, int64_t n, const double* __restrict__ in, double* __restrict__ out);
__global__ void helm_join_vec_kernel(int R, int64_t n, const double* __restrict__ in, double* __restrict__ out);
// near-field assembly (kernels_setup.cu): the streaming form of the regular and
// subdivided pairs, used where the shared-matrix form needs more than
// IBEM_MAX_SMEM_BYTES (near_shared_bytes) of shared memory
cudaError_t launch_near_stream(ibem_handle* h, int cls, bool cplx, double kappa, double* blocks);
// the graded pairs (orders != Q), one streaming launch per (class, order) group
cudaError_t launch_near_graded(ibem_handle* h, bool cplx, double kappa, double* blocks);
size_t near_shared_bytes(int Q, int nb, bool cplx, bool subdiv);
// potential_fmm.cu
cudaError_t launch_potential_fmm(ibem_handle* h, const double* w, int nrhs, const double* pts, int64_t npts,
                                 double* u, int64_t* n_far_terms, int64_t* n_near_terms);
cudaError_t launch_rhs_sources(ibem_handle* h, const double* src, const double* charges, int nrhs, int64_t nsrc,
                               double* b, int64_t* n_far_terms, int64_t* n_near_terms);
// kernels_*.cu entry points (launch on h->stream; return cudaError_t)
cudaError_t launch_geometry_tables(ibem_handle* h);
cudaError_t launch_near_assembly(ibem_handle* h);
cudaError_t launch_far_assembly(ibem_handle* h);
cudaError_t apply_operator(ibem_handle* h, const double* x, double* y, int nrhs, int precision);
cudaError_t launch_rhs(ibem_handle* h, const double* g, int nrhs, double* b);
cudaError_t launch_potential(ibem_handle* h, const double* w, int nrhs, const double* pts,
                             int64_t npts, double* u);
// the direct Laplace potential on caller-provided work space (ws: ndof_super
// doubles, srcs: E Q^2 sources); used by launch_potential and the
// allocation-free entry point
cudaError_t launch_potential_ws(ibem_handle* h, const double* w, int nrhs, const double* pts, int64_t npts,
                                double* u, double* ws, double4_32a* srcs);
cudaError_t launch_near_diagonal(ibem_handle* h, double* diag);
ibem_status solve_impl(ibem_handle* h, const double* b, double* w, int nrhs, double rtol,
                       int maxit, int precond, int precision, ibem_solve_info* info);
// lock-step solver for several right-hand sides (solve_block.cu)
ibem_status solve_block_impl(ibem_handle* h, const double* b, double* x, int R, double rtol, int maxit,
                             int precond, int precision, ibem_solve_info* info);
cudaError_t ensure_workspace(ibem_handle* h, int nrhs);
cudaError_t build_block_jacobi(ibem_handle* h, std::string* err);
bool mr_supported(const ibem_handle* h, int nrhs);
// stored BF16 coupling of the tensor-core path (kernels_mrhs.cu)
bool mr_store_possible(const ibem_handle* h);
cudaError_t mr_store_coupling(ibem_handle* h);
cudaError_t apply_operator_mrhs(ibem_handle* h, const double* x, double* y, int nrhs);
void apply_block_jacobi(ibem_handle* h, const double* r, double* z);
// Helmholtz coupling generated in double-float for many right-hand sides (kernels_gen.cu).
bool gen_supported(const ibem_handle* h);
cudaError_t launch_coupling_gen(ibem_handle* h, int R);
// The same coupling contracted on the tensor cores in BF16 digit slices (q = 8).
bool sliced_supported(const ibem_handle* h);
cudaError_t launch_coupling_sliced(ibem_handle* h, int R);
// Double-float coupling launcher and the autotuner of its ring depth (kernels_apply.cu).
cudaError_t launch_coupling_df(ibem_handle* h, int R, int nst);
cudaError_t tune_coupling_df(ibem_handle* h);

// Learned preconditioner (cnn.cu): z = s + sigma net(s / sigma), s = B^-1 v.
cudaError_t cnn_precondition(ibem_handle* h, ibem_cnn* c, const double* v, double* z);
// Residual/error training pairs from block-Jacobi GMRES solves (solve.cu).
ibem_status solver_pairs_impl(ibem_handle* h, const double* b, int nrhs, double rtol, int maxit, int stride,
                              int max_pairs, float* in_img, float* tgt_img, int* n_pairs, ibem_solve_info* info);
ibem_status solver_residuals_impl(ibem_handle* h, const double* b, int nrhs, double rtol, int maxit, int stride,
                                  int max_vecs, double* r_out, int* n_out, ibem_solve_info* info);
}  // namespace ibem
