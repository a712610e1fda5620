// Setup kernels of libibem (FP64): geometry tables at Gauss and interpolation
// points, near-field Galerkin blocks in the Bernstein superspace, FMM coupling
// matrices, the Jacobi diagonal.
//
// Near field (Sec. 3.2, Sec. 4.3, Sec. 4 item 4): for a near element pair
// (t, s) the block
//     B[i][j] = int_t int_s k(x) k(y) u*(F(x), F(y)) B_i(x) B_j(y) dy dx
// of the (p+1)^2 Bernstein products B_i on each element.  Regular pairs use an
// n x n Gauss rule per element (B = Phi^T G Phi with G[a][b] the weighted
// kernel at Gauss point pairs), subdivided pairs the same on 2 x 2 sub-squares,
// touching pairs the Duffy-type rules of the identical / common-edge /
// common-vertex classes mapped through the pair's canonical orientation.
//
// Coupling (Sec. 4.2): K[a][b] = k(z_a) k(z_b) u*(F(z_a), F(z_b)) at the tensor
// Chebyshev points of the target and source cluster, stored FP64 in the layout
// the apply kernel streams: entry (a, b = s + 4 kk) at [kk][4 a + s].
#include <cstdio>

#include "ibem_internal.cuh"

namespace ibem {

__constant__ double c_gx[IBEM_MAX_GAUSS], c_gw[IBEM_MAX_GAUSS];    // regular Gauss rule on [0, 1]
__constant__ double c_cheb[IBEM_MAX_Q];     // Chebyshev nodes on [0, 1]
__constant__ long long c_level_off[12];

__device__ inline void dev_element_of(int64_t e, int ne1, int* patch, int* ix, int* iy) {
    int64_t per = (int64_t)ne1 * ne1;
    *patch = (int)(e / per);
    uint32_t x, y;
    morton2_inv((uint32_t)(e % per), &x, &y);
    *ix = (int)x;
    *iy = (int)y;
}

__device__ inline void dev_cluster_of(int64_t c, int m, int* patch, int* level, int* ix, int* iy) {
    int l = 0;
    while (l < m && c_level_off[l + 1] <= c) ++l;
    int64_t r = c - c_level_off[l];
    int64_t per = (int64_t)1 << (2 * l);
    *patch = (int)(r / per);
    *level = l;
    uint32_t x, y;
    morton2_inv((uint32_t)(r % per), &x, &y);
    *ix = (int)x;
    *iy = (int)y;
}

// ---- geometry tables -------------------------------------------------------
__global__ void qgeo_kernel(GeomView g, int64_t E, int ne1, int Q, double* qgeo) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int QQ = Q * Q;
    if (idx >= E * QQ) return;
    int64_t e = idx / QQ;
    int gq = (int)(idx % QQ), gx = gq % Q, gy = gq / Q;
    int patch, ix, iy;
    dev_element_of(e, ne1, &patch, &ix, &iy);
    double h = 1.0 / ne1;
    double F[3], Fu[3], Fv[3];
    eval_patch(g, patch, (ix + c_gx[gx]) * h, (iy + c_gx[gy]) * h, F, Fu, Fv);
    double k = surface_measure(Fu, Fv);
    double* o = qgeo + 4 * idx;
    o[0] = F[0]; o[1] = F[1]; o[2] = F[2];
    o[3] = c_gw[gx] * c_gw[gy] * k * h * h;
}

__global__ void igeo_kernel(GeomView g, int64_t C, int m, int q, double* igeo, float* igeo32) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int q2 = q * q;
    if (idx >= C * q2) return;
    int64_t c = idx / q2;
    int a = (int)(idx % q2), au = a % q, av = a / q;
    int patch, level, ix, iy;
    dev_cluster_of(c, m, &patch, &level, &ix, &iy);
    double h = 1.0 / (double)(1 << level);
    double F[3], Fu[3], Fv[3];
    eval_patch(g, patch, (ix + c_cheb[au]) * h, (iy + c_cheb[av]) * h, F, Fu, Fv);
    double k = surface_measure(Fu, Fv);
    double* o = igeo + 4 * idx;
    o[0] = F[0]; o[1] = F[1]; o[2] = F[2]; o[3] = k;
    float* o32 = igeo32 + 4 * idx;
    o32[0] = (float)F[0]; o32[1] = (float)F[1]; o32[2] = (float)F[2]; o32[3] = (float)k;
}

// ---- near field: regular pairs --------------------------------------------
// One CTA per pair.  Shared: XA[QQ][4], XB[QQ][4], G[QQ][QQ], H[QQ][nb].
__global__ void near_regular_kernel(const int32_t* __restrict__ list, int64_t n,
                                    const int32_t* __restrict__ tgt, const int32_t* __restrict__ src,
                                    const double* __restrict__ qgeo, const double* __restrict__ phi,
                                    int QQ, int nb, double* __restrict__ blocks) {
    extern __shared__ double sm[];
    double* XA = sm;
    double* XB = XA + 4 * QQ;
    double* G = XB + 4 * QQ;
    double* H = G + QQ * QQ;
    int64_t k = list[blockIdx.x];
    int64_t t = tgt[k], s = src[k];
    for (int i = threadIdx.x; i < 4 * QQ; i += blockDim.x) {
        XA[i] = qgeo[4 * QQ * t + i];
        XB[i] = qgeo[4 * QQ * s + i];
    }
    __syncthreads();
    const double inv4pi = 1.0 / (4.0 * IBEM_PI);
    for (int i = threadIdx.x; i < QQ * QQ; i += blockDim.x) {
        int a = i / QQ, b = i % QQ;
        double d0 = XA[4 * a] - XB[4 * b], d1 = XA[4 * a + 1] - XB[4 * b + 1], d2 = XA[4 * a + 2] - XB[4 * b + 2];
        double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        G[i] = XA[4 * a + 3] * XB[4 * b + 3] * inv4pi / r;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < QQ * nb; i += blockDim.x) {
        int a = i / nb, j = i % nb;
        double acc = 0.0;
        for (int b = 0; b < QQ; ++b) acc += G[a * QQ + b] * phi[b * nb + j];
        H[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) {
        int r = i / nb, j = i % nb;
        double acc = 0.0;
        for (int a = 0; a < QQ; ++a) acc += phi[a * nb + r] * H[a * nb + j];
        blocks[k * nb * nb + i] = acc;
    }
}

// ---- near field: subdivided pairs (2 x 2 sub-squares of both elements) ------
// Shared: XA[4][QQ][4], XB[4][QQ][4], G[QQ][QQ], H[QQ][nb], acc[nb][nb].
__global__ void near_subdiv_kernel(GeomView g, const int32_t* __restrict__ list, int64_t n,
                                   const int32_t* __restrict__ tgt, const int32_t* __restrict__ src,
                                   const double* __restrict__ phi_sub, int Q, int nb, int ne1,
                                   double* __restrict__ blocks) {
    extern __shared__ double sm[];
    int QQ = Q * Q;
    double* XA = sm;
    double* XB = XA + 16 * QQ;
    double* G = XB + 16 * QQ;
    double* H = G + QQ * QQ;
    double* acc = H + QQ * nb;
    int64_t k = list[blockIdx.x];
    int64_t t = tgt[k], s = src[k];
    double h = 1.0 / ne1;
    for (int i = threadIdx.x; i < 8 * QQ; i += blockDim.x) {
        int which = i / (4 * QQ);      // 0: target, 1: source
        int r = i % (4 * QQ);
        int sub = r / QQ, gq = r % QQ;
        int patch, ix, iy;
        dev_element_of(which ? s : t, ne1, &patch, &ix, &iy);
        double su = 0.5 * (sub & 1) + 0.5 * c_gx[gq % Q];
        double sv = 0.5 * (sub >> 1) + 0.5 * c_gx[gq / Q];
        double F[3], Fu[3], Fv[3];
        eval_patch(g, patch, (ix + su) * h, (iy + sv) * h, F, Fu, Fv);
        double* o = (which ? XB : XA) + 4 * r;
        o[0] = F[0]; o[1] = F[1]; o[2] = F[2];
        o[3] = 0.25 * c_gw[gq % Q] * c_gw[gq / Q] * surface_measure(Fu, Fv) * h * h;
    }
    for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    const double inv4pi = 1.0 / (4.0 * IBEM_PI);
    for (int sa = 0; sa < 4; ++sa)
        for (int sb = 0; sb < 4; ++sb) {
            const double* A = XA + 4 * QQ * sa;
            const double* B = XB + 4 * QQ * sb;
            for (int i = threadIdx.x; i < QQ * QQ; i += blockDim.x) {
                int a = i / QQ, b = i % QQ;
                double d0 = A[4 * a] - B[4 * b], d1 = A[4 * a + 1] - B[4 * b + 1], d2 = A[4 * a + 2] - B[4 * b + 2];
                G[i] = A[4 * a + 3] * B[4 * b + 3] * inv4pi / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            }
            __syncthreads();
            const double* pb = phi_sub + (size_t)sb * QQ * nb;
            for (int i = threadIdx.x; i < QQ * nb; i += blockDim.x) {
                int a = i / nb, j = i % nb;
                double v = 0.0;
                for (int b = 0; b < QQ; ++b) v += G[a * QQ + b] * pb[b * nb + j];
                H[i] = v;
            }
            __syncthreads();
            const double* pa = phi_sub + (size_t)sa * QQ * nb;
            for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) {
                int r = i / nb, j = i % nb;
                double v = 0.0;
                for (int a = 0; a < QQ; ++a) v += pa[a * nb + r] * H[a * nb + j];
                acc[i] += v;
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) blocks[k * nb * nb + i] = acc[i];
}

// ---- near field: regular and subdivided pairs, streaming form -------------
// For Gauss orders whose Q^2 x Q^2 kernel matrix does not fit in shared memory
// (the forms above keep it there).  One CTA of NS_T threads per pair; for each
// pair of point sets (the elements themselves, or each of the 2 x 2 x 2 x 2
// sub-square pairs) the CTA walks the target points in chunks of NS_T: thread t
// forms H[a][j] = sum_b G(a, b) phi_B[b][j] for its target point a in
// registers (G = w_a w_b u*(x_a, y_b), complex for Helmholtz), the chunk is
// stored in shared memory, and the block entries B[r][j] += sum_a phi_A[a][r]
// H[a][j] are accumulated by their owning threads (entry e = t + NS_T i).
// The same sums as the shared-matrix forms, in the same order over b for each
// H[a][j]; the sum over a runs chunk by chunk.  Shared: XA[QQ][4], XB[QQ][4],
// H[NS_T][NB] (real and imaginary parts for Helmholtz).
constexpr int NS_T = 128;

// F and the surface measure at one parameter point, compiled once for all
// instantiations of the streaming kernel (it runs at assembly only)
__device__ __noinline__ void stream_point_geometry(GeomView g, int patch, double u, double v, double* F, double* k) {
    double Fu[3], Fv[3];
    eval_patch(g, patch, u, v, F, Fu, Fv);
    *k = surface_measure(Fu, Fv);
}

template <bool CPLX, int NB>
__global__ void __launch_bounds__(NS_T) near_stream_kernel(GeomView g, const int32_t* __restrict__ list,
                                                           const int32_t* __restrict__ tgt,
                                                           const int32_t* __restrict__ src,
                                                           const double* __restrict__ qgeo,
                                                           const double* __restrict__ phi, int Q, int ne1,
                                                           bool subdiv, double kappa, const double* __restrict__ rule,
                                                           double* __restrict__ blocks) {
    extern __shared__ double sm[];
    constexpr int CW = CPLX ? 2 : 1;
    constexpr int NE = (NB * NB + NS_T - 1) / NS_T;     // block entries per thread
    const int QQ = Q * Q;
    double* XA = sm;
    double* XB = XA + 4 * QQ;
    double* Hr = XB + 4 * QQ;
    double* Hi = Hr + NS_T * NB;
    const int64_t k = list[blockIdx.x];
    const int64_t t = tgt[k], s = src[k];
    const double h = 1.0 / ne1;
    const double inv4pi = 1.0 / (4.0 * IBEM_PI);
    double acc[NE][CW];
#pragma unroll
    for (int i = 0; i < NE; ++i)
#pragma unroll
        for (int c = 0; c < CW; ++c) acc[i][c] = 0.0;
    const int nsub = subdiv ? 4 : 1;
    // rule given (a graded order): nodes rule[0..Q), weights rule[Q..2Q), and the
    // geometry evaluated here; otherwise the module rule and the qgeo table
    const double sc = subdiv ? 0.5 : 1.0;
    for (int sa = 0; sa < nsub; ++sa)
        for (int sb = 0; sb < nsub; ++sb) {
            __syncthreads();   // the previous pass is done with XA, XB and H
            for (int i = threadIdx.x; i < 2 * QQ; i += NS_T) {
                const int which = i / QQ, gq = i % QQ;
                double* o = (which ? XB : XA) + 4 * gq;
                if (!subdiv && !rule) {
                    const double* in = qgeo + 4 * (QQ * (which ? s : t) + gq);
                    o[0] = in[0]; o[1] = in[1]; o[2] = in[2]; o[3] = in[3];
                } else {
                    const int sub = which ? sb : sa;
                    int patch, ix, iy;
                    dev_element_of(which ? s : t, ne1, &patch, &ix, &iy);
                    const double xu = rule ? rule[gq % Q] : c_gx[gq % Q];
                    const double xv = rule ? rule[gq / Q] : c_gx[gq / Q];
                    const double wu = rule ? rule[Q + gq % Q] : c_gw[gq % Q];
                    const double wv = rule ? rule[Q + gq / Q] : c_gw[gq / Q];
                    const double su = sc * (sub & 1) + sc * xu;
                    const double sv = sc * (sub >> 1) + sc * xv;
                    double F[3], k;
                    stream_point_geometry(g, patch, (ix + su) * h, (iy + sv) * h, F, &k);
                    o[0] = F[0]; o[1] = F[1]; o[2] = F[2];
                    o[3] = sc * sc * wu * wv * k * h * h;
                }
            }
            __syncthreads();
            const double* pA = phi + (size_t)(subdiv ? sa : 0) * QQ * NB;
            const double* pB = phi + (size_t)(subdiv ? sb : 0) * QQ * NB;
            for (int a0 = 0; a0 < QQ; a0 += NS_T) {
                const int a = a0 + threadIdx.x;
                double hr[NB], hi[NB];
#pragma unroll
                for (int j = 0; j < NB; ++j) hr[j] = hi[j] = 0.0;
                if (a < QQ) {
                    const double xa0 = XA[4 * a], xa1 = XA[4 * a + 1], xa2 = XA[4 * a + 2], wa = XA[4 * a + 3];
                    for (int b = 0; b < QQ; ++b) {
                        const double d0 = xa0 - XB[4 * b], d1 = xa1 - XB[4 * b + 1], d2 = xa2 - XB[4 * b + 2];
                        const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                        double gr, gi = 0.0;
                        if constexpr (CPLX) {
                            double sn, cs;
                            sincos(kappa * r, &sn, &cs);
                            const double f = wa * XB[4 * b + 3] / (4.0 * IBEM_PI * r);
                            gr = f * cs;
                            gi = f * sn;
                        } else {
                            gr = wa * XB[4 * b + 3] * inv4pi / r;
                        }
                        const double* pb = pB + (size_t)b * NB;
#pragma unroll
                        for (int j = 0; j < NB; ++j) {
                            hr[j] += gr * pb[j];
                            if constexpr (CPLX) hi[j] += gi * pb[j];
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    Hr[threadIdx.x * NB + j] = hr[j];
                    if constexpr (CPLX) Hi[threadIdx.x * NB + j] = hi[j];
                }
                __syncthreads();
                const int na = QQ - a0 < NS_T ? QQ - a0 : NS_T;
#pragma unroll
                for (int i = 0; i < NE; ++i) {
                    const int e = threadIdx.x + NS_T * i;
                    if (e < NB * NB) {
                        const int r = e / NB, j = e % NB;
                        double vr = 0.0, vi = 0.0;
                        for (int aa = 0; aa < na; ++aa) {
                            const double pa = pA[(size_t)(a0 + aa) * NB + r];
                            vr += pa * Hr[aa * NB + j];
                            if constexpr (CPLX) vi += pa * Hi[aa * NB + j];
                        }
                        acc[i][0] += vr;
                        if constexpr (CPLX) acc[i][CW - 1] += vi;
                    }
                }
                __syncthreads();
            }
        }
#pragma unroll
    for (int i = 0; i < NE; ++i) {
        const int e = threadIdx.x + NS_T * i;
        if (e < NB * NB)
#pragma unroll
            for (int c = 0; c < CW; ++c) blocks[(k * NB * NB + e) * CW + c] = acc[i][c];
    }
}

template <bool CPLX>
cudaError_t launch_near_stream_t(ibem_handle* h, int cls, double kappa, double* blocks) {
    Plan& P = h->P;
    GeomView g{h->d_patches, h->d_knots, h->d_cpw};
    const bool subdiv = cls == CLS_SUBDIV;
    const int QQ = P.Q * P.Q;
    const size_t sm = (size_t)(8 * QQ + (CPLX ? 2 : 1) * NS_T * P.nb) * sizeof(double);
    const double* phi = subdiv ? h->d_phi_sub : h->d_phi;
    const unsigned n = (unsigned)h->n_list[cls];
    cudaError_t e;
#define IBEM_NS_CASE(NB_)                                                                                      \
    case NB_:                                                                                                  \
        if ((e = cudaFuncSetAttribute(near_stream_kernel<CPLX, NB_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                      (int)sm)))                                                                \
            return e;                                                                                          \
        near_stream_kernel<CPLX, NB_><<<n, NS_T, sm, h->stream>>>(g, h->d_pairs_by_cls[cls], h->d_near_tgt,     \
                                                                  h->d_near_src, h->d_qgeo, phi, P.Q, P.ne1,    \
                                                                  subdiv, kappa, nullptr, blocks);              \
        break;
    switch (P.nb) {
        IBEM_NS_CASE(1)
        IBEM_NS_CASE(4)
        IBEM_NS_CASE(9)
        IBEM_NS_CASE(16)
        IBEM_NS_CASE(25)
        default: return cudaErrorInvalidValue;
    }
#undef IBEM_NS_CASE
    return cudaGetLastError();
}

// Graded pairs: one streaming launch per (class, order) group, each with its
// own rule and Bernstein table.
template <bool CPLX>
cudaError_t launch_near_graded_t(ibem_handle* h, double kappa, double* blocks) {
    Plan& P = h->P;
    GeomView g{h->d_patches, h->d_knots, h->d_cpw};
    cudaError_t e;
    for (const auto& gr : h->graded) {
        const int Q = gr.order, QQ = Q * Q;
        const bool subdiv = gr.cls == CLS_SUBDIV;
        const size_t sm = (size_t)(8 * QQ + (CPLX ? 2 : 1) * NS_T * P.nb) * sizeof(double);
        if (sm > IBEM_MAX_SMEM_BYTES) return cudaErrorInvalidValue;
        const double* rule = h->d_graded_tab + gr.tab_off;
        const double* phi = rule + 2 * Q;
        const int32_t* list = h->d_graded_pairs + gr.off;
        const unsigned n = (unsigned)gr.count;
#define IBEM_NG_CASE(NB_)                                                                                        \
    case NB_:                                                                                                    \
        if ((e = cudaFuncSetAttribute(near_stream_kernel<CPLX, NB_>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                      (int)sm)))                                                                  \
            return e;                                                                                            \
        near_stream_kernel<CPLX, NB_><<<n, NS_T, sm, h->stream>>>(g, list, h->d_near_tgt, h->d_near_src, nullptr, \
                                                                  phi, Q, P.ne1, subdiv, kappa, rule, blocks);    \
        break;
        switch (P.nb) {
            IBEM_NG_CASE(1)
            IBEM_NG_CASE(4)
            IBEM_NG_CASE(9)
            IBEM_NG_CASE(16)
            IBEM_NG_CASE(25)
            default: return cudaErrorInvalidValue;
        }
#undef IBEM_NG_CASE
        if ((e = cudaGetLastError())) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_near_graded(ibem_handle* h, bool cplx, double kappa, double* blocks) {
    if (h->graded.empty()) return cudaSuccess;
    return cplx ? launch_near_graded_t<true>(h, kappa, blocks) : launch_near_graded_t<false>(h, kappa, blocks);
}

cudaError_t launch_near_stream(ibem_handle* h, int cls, bool cplx, double kappa, double* blocks) {
    cudaError_t e;
    std::vector<double> gx, gw;
    gauss_legendre(h->P.Q, gx, gw);
    if ((e = cudaMemcpyToSymbolAsync(c_gx, gx.data(), h->P.Q * sizeof(double), 0, cudaMemcpyHostToDevice, h->stream)) ||
        (e = cudaMemcpyToSymbolAsync(c_gw, gw.data(), h->P.Q * sizeof(double), 0, cudaMemcpyHostToDevice, h->stream)))
        return e;
    return cplx ? launch_near_stream_t<true>(h, cls, kappa, blocks) : launch_near_stream_t<false>(h, cls, kappa, blocks);
}

size_t near_shared_bytes(int Q, int nb, bool cplx, bool subdiv) {
    const size_t QQ = (size_t)Q * Q, cw = cplx ? 2 : 1;
    return (subdiv ? 32 * QQ + cw * QQ * QQ + cw * QQ * nb + cw * nb * nb : 8 * QQ + cw * QQ * QQ + cw * QQ * nb) *
           sizeof(double);
}

// ---- near field: touching pairs (Duffy-type rules) -------------------------
// The rule's canonical points (x^, y^) are mapped by rho_{kA} and rho_{kB} into
// the element-local squares.  Points are processed in chunks of blockDim.x.
// Shared: SA[nb][CH], SB[nb][CH].
__global__ void near_singular_kernel(GeomView g, const int32_t* __restrict__ list, int64_t n,
                                     const int32_t* __restrict__ tgt, const int32_t* __restrict__ src,
                                     const int32_t* __restrict__ orient, const double* __restrict__ rule,
                                     int npts, int p, int ne1, double* __restrict__ blocks) {
    extern __shared__ double sm[];
    const int CH = blockDim.x;
    const int pp = p + 1, nb = pp * pp;
    double* SA = sm;
    double* SB = SA + nb * CH;
    int64_t k = list[blockIdx.x];
    int64_t t = tgt[k], s = src[k];
    int ka = orient[k] >> 3, kb = orient[k] & 7;
    int pa, ixa, iya, pb, ixb, iyb;
    dev_element_of(t, ne1, &pa, &ixa, &iya);
    dev_element_of(s, ne1, &pb, &ixb, &iyb);
    double h = 1.0 / ne1;
    const double scale = h * h * h * h / (4.0 * IBEM_PI);
    double acc[5] = {0, 0, 0, 0, 0};   // nb * nb <= 625 <= 5 * 128 entries per thread
    for (int base = 0; base < npts; base += CH) {
        int ip = base + threadIdx.x;
        if (ip < npts) {
            double x1 = rule[ip], x2 = rule[npts + ip], y1 = rule[2 * npts + ip], y2 = rule[3 * npts + ip];
            double w = rule[4 * npts + ip];
            double xa, ya, xb, yb;
            dihedral(ka, x1, x2, &xa, &ya);
            dihedral(kb, y1, y2, &xb, &yb);
            double FA[3], FB[3], Fu[3], Fv[3];
            eval_patch(g, pa, (ixa + xa) * h, (iya + ya) * h, FA, Fu, Fv);
            double kA = surface_measure(Fu, Fv);
            eval_patch(g, pb, (ixb + xb) * h, (iyb + yb) * h, FB, Fu, Fv);
            double kB = surface_measure(Fu, Fv);
            double d0 = FA[0] - FB[0], d1 = FA[1] - FB[1], d2 = FA[2] - FB[2];
            double val = w * scale * kA * kB / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            double bxu[IBEM_MAX_P + 1], bxv[IBEM_MAX_P + 1], byu[IBEM_MAX_P + 1], byv[IBEM_MAX_P + 1];
            bernstein(p, xa, bxu);
            bernstein(p, ya, bxv);
            bernstein(p, xb, byu);
            bernstein(p, yb, byv);
            for (int iv = 0; iv < pp; ++iv)
                for (int iu = 0; iu < pp; ++iu) {
                    SA[(iv * pp + iu) * CH + threadIdx.x] = val * bxu[iu] * bxv[iv];
                    SB[(iv * pp + iu) * CH + threadIdx.x] = byu[iu] * byv[iv];
                }
        } else {
            for (int i = 0; i < nb; ++i) {
                SA[i * CH + threadIdx.x] = 0.0;
                SB[i * CH + threadIdx.x] = 0.0;
            }
        }
        __syncthreads();
        for (int r = 0; r < 5; ++r) {
            int e = threadIdx.x + r * CH;
            if (e < nb * nb) {
                int i = e / nb, j = e % nb;
                const double* a = SA + i * CH;
                const double* b = SB + j * CH;
                double v = 0.0;
                for (int c = 0; c < CH; ++c) v += a[c] * b[c];
                acc[r] += v;
            }
        }
        __syncthreads();
    }
    for (int r = 0; r < 5; ++r) {
        int e = threadIdx.x + r * CH;
        if (e < nb * nb) blocks[k * nb * nb + e] = acc[r];
    }
}

// ---- far field: coupling matrices -----------------------------------------
// Stored as doubles (native) or as float pairs hi = fl(K), lo = fl(K - hi).
__global__ void far_assemble_kernel(int64_t n_far, const int32_t* __restrict__ ftgt,
                                    const int32_t* __restrict__ fsrc, const double* __restrict__ igeo,
                                    int q2, int kpt, double* __restrict__ K, float2* __restrict__ Kdf) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t per = (int64_t)kpt * 4 * q2;
    if (idx >= n_far * per) return;
    int64_t blk = idx / per;
    int r = (int)(idx % per);
    int kk = r / (4 * q2), t = r % (4 * q2);
    int a = t >> 2, s = t & 3, b = s + 4 * kk;
    double v = 0.0;
    if (b < q2) {
        const double* A = igeo + 4 * ((int64_t)ftgt[blk] * q2 + a);
        const double* B = igeo + 4 * ((int64_t)fsrc[blk] * q2 + b);
        double d0 = A[0] - B[0], d1 = A[1] - B[1], d2 = A[2] - B[2];
        v = A[3] * B[3] / (4.0 * IBEM_PI * sqrt(d0 * d0 + d1 * d1 + d2 * d2));
    }
    if (K) {
        K[idx] = v;
    } else {
        float hi = (float)v;
        Kdf[idx] = make_float2(hi, (float)(v - (double)hi));
    }
}

// ---- Jacobi diagonal of T A_near T^T ---------------------------------------
// For dof (patch, ju, jv): sum over element pairs (e, e') in its support that
// are near pairs of T[dof, (e, i)] B_{e e'}[i][i'] T[dof, (e', i')].
__global__ void near_diag_kernel(int64_t N, int npatch, int p, int ne1, const int64_t* __restrict__ nptr,
                                 const int32_t* __restrict__ nsrc, const double* __restrict__ blocks,
                                 const double* __restrict__ ext, double* __restrict__ diag) {
    int64_t dof = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (dof >= N) return;
    int pp = p + 1, nb = pp * pp, n1 = ne1 + p;
    int patch = (int)(dof / ((int64_t)n1 * n1));
    int rem = (int)(dof % ((int64_t)n1 * n1));
    int jv = rem / n1, ju = rem % n1;
    int64_t per = (int64_t)ne1 * ne1;
    double acc = 0.0;
    for (int iy = jv - p; iy <= jv; ++iy)
        for (int ix = ju - p; ix <= ju; ++ix) {
            if (ix < 0 || iy < 0 || ix >= ne1 || iy >= ne1) continue;
            int64_t e = patch * per + morton2(ix, iy);
            const double* cu = ext + ((int64_t)ix * pp + (ju - ix)) * pp;
            const double* cv = ext + ((int64_t)iy * pp + (jv - iy)) * pp;
            for (int iy2 = jv - p; iy2 <= jv; ++iy2)
                for (int ix2 = ju - p; ix2 <= ju; ++ix2) {
                    if (ix2 < 0 || iy2 < 0 || ix2 >= ne1 || iy2 >= ne1) continue;
                    int64_t e2 = patch * per + morton2(ix2, iy2);
                    // binary search e2 in the sorted sources of row e
                    int64_t lo = nptr[e], hi = nptr[e + 1];
                    while (lo < hi) {
                        int64_t mid = (lo + hi) >> 1;
                        if (nsrc[mid] < e2) lo = mid + 1; else hi = mid;
                    }
                    if (lo >= nptr[e + 1] || nsrc[lo] != e2) continue;
                    const double* B = blocks + lo * nb * nb;
                    const double* du = ext + ((int64_t)ix2 * pp + (ju - ix2)) * pp;
                    const double* dv = ext + ((int64_t)iy2 * pp + (jv - iy2)) * pp;
                    for (int i = 0; i < nb; ++i) {
                        double ti = cu[i % pp] * cv[i / pp];
                        double row = 0.0;
                        for (int j = 0; j < nb; ++j) row += B[i * nb + j] * du[j % pp] * dv[j / pp];
                        acc += ti * row;
                    }
                }
        }
    diag[dof] = acc;
}

__global__ void to_float_kernel(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}


static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_geometry_tables(ibem_handle* h) {
    Plan& P = h->P;
    std::vector<double> gx, gw;
    gauss_legendre(P.Q, gx, gw);
    cudaError_t e;
    if ((e = cudaMemcpyToSymbolAsync(c_gx, gx.data(), P.Q * sizeof(double), 0, cudaMemcpyHostToDevice, h->stream))) return e;
    if ((e = cudaMemcpyToSymbolAsync(c_gw, gw.data(), P.Q * sizeof(double), 0, cudaMemcpyHostToDevice, h->stream))) return e;
    long long lo[12] = {0};
    for (size_t l = 0; l < P.level_off.size() && l < 12; ++l) lo[l] = P.level_off[l];
    if ((e = cudaMemcpyToSymbolAsync(c_level_off, lo, sizeof(lo), 0, cudaMemcpyHostToDevice, h->stream))) return e;
    GeomView g{h->d_patches, h->d_knots, h->d_cpw};
    int QQ = P.Q * P.Q;
    qgeo_kernel<<<nblk(P.E * QQ, 128), 128, 0, h->stream>>>(g, P.E, P.ne1, P.Q, h->d_qgeo);
    if (P.q > 0) {
        std::vector<double> z;
        chebyshev_nodes(P.q, z);
        if ((e = cudaMemcpyToSymbolAsync(c_cheb, z.data(), P.q * sizeof(double), 0, cudaMemcpyHostToDevice, h->stream))) return e;
        igeo_kernel<<<nblk(P.C * P.q2, 128), 128, 0, h->stream>>>(g, P.C, P.m, P.q, h->d_igeo, h->d_igeo32);
    }
    return cudaGetLastError();
}

cudaError_t launch_near_assembly(ibem_handle* h) {
    Plan& P = h->P;
    GeomView g{h->d_patches, h->d_knots, h->d_cpw};
    int QQ = P.Q * P.Q, nb = P.nb;
    cudaError_t e;
    // the Gauss rule is module-wide: load this handle's before the subdivided pairs use it
    {
        std::vector<double> gx, gw;
        gauss_legendre(P.Q, gx, gw);
        if ((e = cudaMemcpyToSymbolAsync(c_gx, gx.data(), P.Q * sizeof(double), 0, cudaMemcpyHostToDevice,
                                         h->stream)) ||
            (e = cudaMemcpyToSymbolAsync(c_gw, gw.data(), P.Q * sizeof(double), 0, cudaMemcpyHostToDevice,
                                         h->stream)))
            return e;
    }
    for (int cls : {CLS_REGULAR, CLS_SUBDIV}) {
        if (h->n_list[cls] > 0 && near_shared_bytes(P.Q, nb, false, cls == CLS_SUBDIV) > IBEM_MAX_SMEM_BYTES &&
            (e = launch_near_stream(h, cls, false, 0.0, h->d_near)))
            return e;
    }
    if ((e = launch_near_graded(h, false, 0.0, h->d_near))) return e;
    // regular
    if (h->n_list[CLS_REGULAR] > 0 && near_shared_bytes(P.Q, nb, false, false) <= IBEM_MAX_SMEM_BYTES) {
        size_t sm = (size_t)(8 * QQ + QQ * QQ + QQ * nb) * sizeof(double);
        if ((e = cudaFuncSetAttribute(near_regular_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
        near_regular_kernel<<<(unsigned)h->n_list[CLS_REGULAR], 128, sm, h->stream>>>(
            h->d_pairs_by_cls[CLS_REGULAR], h->n_list[CLS_REGULAR], h->d_near_tgt, h->d_near_src, h->d_qgeo,
            h->d_phi, QQ, nb, h->d_near);
    }
    if (h->n_list[CLS_SUBDIV] > 0 && near_shared_bytes(P.Q, nb, false, true) <= IBEM_MAX_SMEM_BYTES) {
        size_t sm = (size_t)(32 * QQ + QQ * QQ + QQ * nb + nb * nb) * sizeof(double);
        if ((e = cudaFuncSetAttribute(near_subdiv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
        near_subdiv_kernel<<<(unsigned)h->n_list[CLS_SUBDIV], 128, sm, h->stream>>>(
            g, h->d_pairs_by_cls[CLS_SUBDIV], h->n_list[CLS_SUBDIV], h->d_near_tgt, h->d_near_src, h->d_phi_sub,
            P.Q, nb, P.ne1, h->d_near);
    }
    for (int c = 0; c < 3; ++c) {
        if (h->n_list[c] == 0) continue;
        const int CH = 128;
        size_t sm = (size_t)2 * nb * CH * sizeof(double);
        if ((e = cudaFuncSetAttribute(near_singular_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
        near_singular_kernel<<<(unsigned)h->n_list[c], CH, sm, h->stream>>>(
            g, h->d_pairs_by_cls[c], h->n_list[c], h->d_near_tgt, h->d_near_src, h->d_near_orient, h->d_rule[c],
            h->rule_n[c], P.p, P.ne1, h->d_near);
    }
    if ((e = cudaGetLastError())) return e;
    int64_t nn = P.n_near * nb * nb;
    to_float_kernel<<<nblk(nn, 256), 256, 0, h->stream>>>(h->d_near, h->d_near32, nn);
    near_diag_kernel<<<nblk(P.N, 128), 128, 0, h->stream>>>(P.N, P.npatch, P.p, P.ne1, h->d_near_ptr,
                                                            h->d_near_src, h->d_near, h->d_ext, h->d_diag);
    return cudaGetLastError();
}

cudaError_t launch_far_assembly(ibem_handle* h) {
    Plan& P = h->P;
    // nothing stored (IBEM_COUPLING_NONE) or no far field: nothing to assemble
    if (P.n_far == 0 || (!h->d_K && !h->d_Kdf)) return cudaSuccess;
    // native: every far block; double-float: the upper half (symmetric storage)
    const bool native = h->d_K != nullptr;
    const int64_t nblocks = native ? P.n_far : h->n_up;
    if (nblocks == 0) return cudaSuccess;
    int64_t total = nblocks * (int64_t)h->kpt * 4 * P.q2;
    far_assemble_kernel<<<nblk(total, 256), 256, 0, h->stream>>>(nblocks, native ? h->d_far_tgt : h->d_up_tgt,
                                                                 native ? h->d_far_src : h->d_up_src, h->d_igeo,
                                                                 P.q2, h->kpt, h->d_K, h->d_Kdf);
    return cudaGetLastError();
}

}  // namespace ibem
