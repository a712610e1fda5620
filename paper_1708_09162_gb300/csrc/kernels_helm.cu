// Helmholtz (complex) parts of libibem.  Fundamental solution
// u*(x, y) = exp(i kappa |x - y|) / (4 pi |x - y|) (Eq. fundament2); the bilinear
// form has no conjugation, so every block is complex-symmetric.
//
// Layout: the public complex arrays are interleaved (re, im).  Inside an
// application they are split into 2R real right-hand sides (index 2r for the
// real part, 2r + 1 for the imaginary part), so every step whose coefficients
// are real (T^T, moments, M2M, L2L, back-projection, T) runs the real kernels
// unchanged; only the near product and the coupling mix real and imaginary
// parts.
//
// Near blocks: [n_near][nb][nb] double2 (re, im).  Coupling matrices of the
// FP64 operator: stored as double-float complex (re_hi, re_lo, im_hi, im_lo),
// layout [n_far][kpt][4 q2] like the Laplace case, or - when they would not fit
// in the memory budget - generated on the fly in FP64.
#include "ibem_internal.cuh"

namespace ibem {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__constant__ double c_hgx[IBEM_MAX_GAUSS], c_hgw[IBEM_MAX_GAUSS];

__device__ inline void helm_elem(int64_t e, int ne1, int* patch, int* ix, int* iy) {
    int64_t per = (int64_t)ne1 * ne1;
    *patch = (int)(e / per);
    uint32_t x, y;
    morton2_inv((uint32_t)(e % per), &x, &y);
    *ix = (int)x;
    *iy = (int)y;
}

// exp(i kappa r) / (4 pi r) * w
__device__ inline void helm_kernel64(double kappa, double r, double w, double* re, double* im) {
    double s, c;
    sincos(kappa * r, &s, &c);
    double f = w / (4.0 * IBEM_PI * r);
    *re = f * c;
    *im = f * s;
}

// ---- near field assembly -------------------------------------------------------
// Regular pairs: one CTA per pair; shared XA[QQ][4], XB[QQ][4], Gre, Gim [QQ][QQ],
// Hre, Him [QQ][nb].
__global__ void helm_near_regular_kernel(const int32_t* __restrict__ list, const int32_t* __restrict__ tgt,
                                         const int32_t* __restrict__ src, const double* __restrict__ qgeo,
                                         const double* __restrict__ phi, int QQ, int nb, double kappa,
                                         double2* __restrict__ blocks) {
    extern __shared__ double sm[];
    double* XA = sm;
    double* XB = XA + 4 * QQ;
    double* Gr = XB + 4 * QQ;
    double* Gi = Gr + QQ * QQ;
    double* Hr = Gi + QQ * QQ;
    double* Hi = Hr + QQ * nb;
    int64_t k = list[blockIdx.x];
    int64_t t = tgt[k], s = src[k];
    for (int i = threadIdx.x; i < 4 * QQ; i += blockDim.x) {
        XA[i] = qgeo[4 * QQ * t + i];
        XB[i] = qgeo[4 * QQ * s + i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < QQ * QQ; i += blockDim.x) {
        int a = i / QQ, b = i % QQ;
        double d0 = XA[4 * a] - XB[4 * b], d1 = XA[4 * a + 1] - XB[4 * b + 1], d2 = XA[4 * a + 2] - XB[4 * b + 2];
        helm_kernel64(kappa, sqrt(d0 * d0 + d1 * d1 + d2 * d2), XA[4 * a + 3] * XB[4 * b + 3], &Gr[i], &Gi[i]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < QQ * nb; i += blockDim.x) {
        int a = i / nb, j = i % nb;
        double vr = 0.0, vi = 0.0;
        for (int b = 0; b < QQ; ++b) {
            double p = phi[b * nb + j];
            vr += Gr[a * QQ + b] * p;
            vi += Gi[a * QQ + b] * p;
        }
        Hr[i] = vr;
        Hi[i] = vi;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) {
        int r = i / nb, j = i % nb;
        double vr = 0.0, vi = 0.0;
        for (int a = 0; a < QQ; ++a) {
            double p = phi[a * nb + r];
            vr += p * Hr[a * nb + j];
            vi += p * Hi[a * nb + j];
        }
        blocks[k * nb * nb + i] = make_double2(vr, vi);
    }
}

// Subdivided pairs: 2 x 2 sub-squares of both elements, geometry on the fly.
__global__ void helm_near_subdiv_kernel(GeomView g, const int32_t* __restrict__ list, const int32_t* __restrict__ tgt,
                                        const int32_t* __restrict__ src, const double* __restrict__ phi_sub, int Q,
                                        int nb, int ne1, double kappa, double2* __restrict__ blocks) {
    extern __shared__ double sm[];
    int QQ = Q * Q;
    double* XA = sm;
    double* XB = XA + 16 * QQ;
    double* Gr = XB + 16 * QQ;
    double* Gi = Gr + QQ * QQ;
    double* Hr = Gi + QQ * QQ;
    double* Hi = Hr + QQ * nb;
    double* ar = Hi + QQ * nb;
    double* ai = ar + nb * nb;
    int64_t k = list[blockIdx.x];
    int64_t t = tgt[k], s = src[k];
    double h = 1.0 / ne1;
    for (int i = threadIdx.x; i < 8 * QQ; i += blockDim.x) {
        int which = i / (4 * QQ);
        int r = i % (4 * QQ);
        int sub = r / QQ, gq = r % QQ;
        int patch, ix, iy;
        helm_elem(which ? s : t, ne1, &patch, &ix, &iy);
        double su = 0.5 * (sub & 1) + 0.5 * c_hgx[gq % Q];
        double sv = 0.5 * (sub >> 1) + 0.5 * c_hgx[gq / Q];
        double F[3], Fu[3], Fv[3];
        eval_patch(g, patch, (ix + su) * h, (iy + sv) * h, F, Fu, Fv);
        double* o = (which ? XB : XA) + 4 * r;
        o[0] = F[0]; o[1] = F[1]; o[2] = F[2];
        o[3] = 0.25 * c_hgw[gq % Q] * c_hgw[gq / Q] * surface_measure(Fu, Fv) * h * h;
    }
    for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) { ar[i] = 0.0; ai[i] = 0.0; }
    __syncthreads();
    for (int sa = 0; sa < 4; ++sa)
        for (int sb = 0; sb < 4; ++sb) {
            const double* A = XA + 4 * QQ * sa;
            const double* B = XB + 4 * QQ * sb;
            for (int i = threadIdx.x; i < QQ * QQ; i += blockDim.x) {
                int a = i / QQ, b = i % QQ;
                double d0 = A[4 * a] - B[4 * b], d1 = A[4 * a + 1] - B[4 * b + 1], d2 = A[4 * a + 2] - B[4 * b + 2];
                helm_kernel64(kappa, sqrt(d0 * d0 + d1 * d1 + d2 * d2), A[4 * a + 3] * B[4 * b + 3], &Gr[i], &Gi[i]);
            }
            __syncthreads();
            const double* pb = phi_sub + (size_t)sb * QQ * nb;
            for (int i = threadIdx.x; i < QQ * nb; i += blockDim.x) {
                int a = i / nb, j = i % nb;
                double vr = 0.0, vi = 0.0;
                for (int b = 0; b < QQ; ++b) {
                    double p = pb[b * nb + j];
                    vr += Gr[a * QQ + b] * p;
                    vi += Gi[a * QQ + b] * p;
                }
                Hr[i] = vr;
                Hi[i] = vi;
            }
            __syncthreads();
            const double* pa = phi_sub + (size_t)sa * QQ * nb;
            for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) {
                int r = i / nb, j = i % nb;
                double vr = 0.0, vi = 0.0;
                for (int a = 0; a < QQ; ++a) {
                    double p = pa[a * nb + r];
                    vr += p * Hr[a * nb + j];
                    vi += p * Hi[a * nb + j];
                }
                ar[i] += vr;
                ai[i] += vi;
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) blocks[k * nb * nb + i] = make_double2(ar[i], ai[i]);
}

// Touching pairs: the Duffy-type rules mapped through the canonical orientation.
// Shared: SAr[nb][CH], SAi[nb][CH], SB[nb][CH].
__global__ void helm_near_singular_kernel(GeomView g, const int32_t* __restrict__ list,
                                          const int32_t* __restrict__ tgt, const int32_t* __restrict__ src,
                                          const int32_t* __restrict__ orient, const double* __restrict__ rule,
                                          int npts, int p, int ne1, double kappa, double2* __restrict__ blocks) {
    extern __shared__ double sm[];
    const int CH = blockDim.x;
    const int pp = p + 1, nb = pp * pp;
    double* SAr = sm;
    double* SAi = SAr + nb * CH;
    double* SB = SAi + nb * CH;
    int64_t k = list[blockIdx.x];
    int64_t t = tgt[k], s = src[k];
    int ka = orient[k] >> 3, kb = orient[k] & 7;
    int pa, ixa, iya, pb, ixb, iyb;
    helm_elem(t, ne1, &pa, &ixa, &iya);
    helm_elem(s, ne1, &pb, &ixb, &iyb);
    double h = 1.0 / ne1;
    const double scale = h * h * h * h;
    double accr[5] = {0, 0, 0, 0, 0}, acci[5] = {0, 0, 0, 0, 0};
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
            double vr, vi;
            helm_kernel64(kappa, sqrt(d0 * d0 + d1 * d1 + d2 * d2), w * scale * kA * kB, &vr, &vi);
            double bxu[IBEM_MAX_P + 1], bxv[IBEM_MAX_P + 1], byu[IBEM_MAX_P + 1], byv[IBEM_MAX_P + 1];
            bernstein(p, xa, bxu);
            bernstein(p, ya, bxv);
            bernstein(p, xb, byu);
            bernstein(p, yb, byv);
            for (int iv = 0; iv < pp; ++iv)
                for (int iu = 0; iu < pp; ++iu) {
                    double ba = bxu[iu] * bxv[iv];
                    SAr[(iv * pp + iu) * CH + threadIdx.x] = vr * ba;
                    SAi[(iv * pp + iu) * CH + threadIdx.x] = vi * ba;
                    SB[(iv * pp + iu) * CH + threadIdx.x] = byu[iu] * byv[iv];
                }
        } else {
            for (int i = 0; i < nb; ++i) {
                SAr[i * CH + threadIdx.x] = 0.0;
                SAi[i * CH + threadIdx.x] = 0.0;
                SB[i * CH + threadIdx.x] = 0.0;
            }
        }
        __syncthreads();
        for (int r = 0; r < 5; ++r) {
            int e = threadIdx.x + r * CH;
            if (e < nb * nb) {
                int i = e / nb, j = e % nb;
                const double* ar = SAr + i * CH;
                const double* ai = SAi + i * CH;
                const double* b = SB + j * CH;
                double vr = 0.0, vi = 0.0;
                for (int c = 0; c < CH; ++c) {
                    vr += ar[c] * b[c];
                    vi += ai[c] * b[c];
                }
                accr[r] += vr;
                acci[r] += vi;
            }
        }
        __syncthreads();
    }
    for (int r = 0; r < 5; ++r) {
        int e = threadIdx.x + r * CH;
        if (e < nb * nb) blocks[k * nb * nb + e] = make_double2(accr[r], acci[r]);
    }
}

__global__ void helm_to_float_kernel(const double2* __restrict__ in, float2* __restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// Jacobi diagonal (complex) of T A_near T^T
__global__ void helm_near_diag_kernel(int64_t N, int p, int ne1, const int64_t* __restrict__ nptr,
                                      const int32_t* __restrict__ nsrc, const double2* __restrict__ blocks,
                                      const double* __restrict__ ext, double2* __restrict__ diag) {
    int64_t dof = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (dof >= N) return;
    int pp = p + 1, nb = pp * pp, n1 = ne1 + p;
    int patch = (int)(dof / ((int64_t)n1 * n1));
    int rem = (int)(dof % ((int64_t)n1 * n1));
    int jv = rem / n1, ju = rem % n1;
    int64_t per = (int64_t)ne1 * ne1;
    double accr = 0.0, acci = 0.0;
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
                    int64_t lo = nptr[e], hi = nptr[e + 1];
                    while (lo < hi) {
                        int64_t mid = (lo + hi) >> 1;
                        if (nsrc[mid] < e2) lo = mid + 1; else hi = mid;
                    }
                    if (lo >= nptr[e + 1] || nsrc[lo] != e2) continue;
                    const double2* B = blocks + lo * nb * nb;
                    const double* du = ext + ((int64_t)ix2 * pp + (ju - ix2)) * pp;
                    const double* dv = ext + ((int64_t)iy2 * pp + (jv - iy2)) * pp;
                    for (int i = 0; i < nb; ++i) {
                        double ti = cu[i % pp] * cv[i / pp];
                        double rr = 0.0, ri = 0.0;
                        for (int j = 0; j < nb; ++j) {
                            double tj = du[j % pp] * dv[j / pp];
                            rr += B[i * nb + j].x * tj;
                            ri += B[i * nb + j].y * tj;
                        }
                        accr += ti * rr;
                        acci += ti * ri;
                    }
                }
        }
    diag[dof] = make_double2(accr, acci);
}

// ---- coupling matrices (stored, double-float complex) ------------------------------
__global__ void helm_far_assemble_kernel(int64_t n_far, const int32_t* __restrict__ ftgt,
                                         const int32_t* __restrict__ fsrc, const double* __restrict__ igeo, int q2,
                                         int kpt, double kappa, float4* __restrict__ K) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t per = (int64_t)kpt * 4 * q2;
    if (idx >= n_far * per) return;
    int64_t blk = idx / per;
    int r = (int)(idx % per);
    int kk = r / (4 * q2), t = r % (4 * q2);
    int a = t >> 2, s = t & 3, b = s + 4 * kk;
    double vr = 0.0, vi = 0.0;
    if (b < q2) {
        const double* A = igeo + 4 * ((int64_t)ftgt[blk] * q2 + a);
        const double* B = igeo + 4 * ((int64_t)fsrc[blk] * q2 + b);
        double d0 = A[0] - B[0], d1 = A[1] - B[1], d2 = A[2] - B[2];
        helm_kernel64(kappa, sqrt(d0 * d0 + d1 * d1 + d2 * d2), A[3] * B[3], &vr, &vi);
    }
    float rh = (float)vr, ih = (float)vi;
    K[idx] = make_float4(rh, (float)(vr - (double)rh), ih, (float)(vi - (double)ih));
}

// split moments of the 2R real "right-hand sides" into double-float complex
// (re_hi, re_lo, im_hi, im_lo) rows of q2p entries (q2p even: 32-byte rows)
__global__ void helm_split_kernel(int R, int64_t C, int q2, int q2p, const double* __restrict__ xh,
                                  float4* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)R * C * q2p) return;
    int64_t r = i / (C * q2p);
    int64_t rem = i % (C * q2p);
    int64_t c = rem / q2p;
    int a = (int)(rem % q2p);
    double vr = 0.0, vi = 0.0;
    if (a < q2) {
        vr = xh[((2 * r) * C + c) * q2 + a];
        vi = xh[((2 * r + 1) * C + c) * q2 + a];
    }
    float rh = (float)vr, ih = (float)vi;
    out[i] = make_float4(rh, (float)(vr - (double)rh), ih, (float)(vi - (double)ih));
}

// double-float helpers: exact product a*b = p + e; acc (hi, lo) += (p, e)
__device__ inline void df_mac(float ah, float al, float bh, float bl, float& hi, float& lo) {
    float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    float t = hi + p;
    float z = t - hi;
    float err = (hi - (t - z)) + (p - z);
    hi = t;
    lo += err + e;
}

__device__ inline unsigned hsmem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ inline void hmbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(hsmem(bar)), "r"(count) : "memory");
}
__device__ inline void hmbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(hsmem(bar)), "r"(bytes) : "memory");
}
__device__ inline void hbulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     hsmem(dst)),
                 "l"(src), "r"(bytes), "r"(hsmem(bar))
                 : "memory");
}
__device__ inline bool hmbar_wait(uint64_t* bar, unsigned parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(hsmem(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Streaming complex coupling, FP64-accurate (double-float), same pipeline as
// the Laplace kernel: one CTA per target cluster, NST stages of (K block,
// source moments) filled by cp.async.bulk, bounded mbarrier waits.
template <int KPT, int NST>
__global__ void helm_coupling_df_kernel(const int32_t* __restrict__ rows, const int64_t* __restrict__ fptr,
                                        const int32_t* __restrict__ fsrc, const float4* __restrict__ K, int q2,
                                        int q2p, int maxrow, int64_t C, const float4* __restrict__ xh,
                                        double* __restrict__ yh, long long wait_limit, int* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    int32_t* srcs = reinterpret_cast<int32_t*>(smem + 128);
    const int stride = 4 * q2;
    const int belems = KPT * stride;
    const int selems = belems + q2p;
    float4* stage = reinterpret_cast<float4*>(smem + 128 + (((size_t)maxrow * 4 + 15) / 16) * 16);
    const unsigned kbytes = (unsigned)belems * 16u, xbytes = (unsigned)q2p * 16u;
    const int sigma = rows[blockIdx.x];
    const int64_t r = blockIdx.y;
    const int t = threadIdx.x, s = t & 3, a = t >> 2;
    const bool active = t < stride;
    const int64_t b0 = fptr[sigma];
    const int n = (int)(fptr[sigma + 1] - b0);
    const float4* xr = xh + r * C * q2p;
    for (int j = t; j < n; j += blockDim.x) srcs[j] = fsrc[b0 + j];
    if (t == 0) {
        for (int i = 0; i < NST; ++i) hmbar_init(&full[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (t == 0) {
        for (int i = 0; i < NST && i < n; ++i) {
            float4* dst = stage + (size_t)i * selems;
            hmbar_expect_tx(&full[i], kbytes + xbytes);
            hbulk_load(dst, K + (b0 + i) * (int64_t)belems, kbytes, &full[i]);
            hbulk_load(dst + belems, xr + (int64_t)srcs[i] * q2p, xbytes, &full[i]);
        }
    }
    double accr = 0.0, acci = 0.0;
    int i = 0;
    bool failed = false;
    for (; i < n; ++i) {
        const int st = i % NST;
        const bool ok = hmbar_wait(&full[st], (unsigned)((i / NST) & 1), wait_limit);
        if (ok && active) {
            const float4* Kb = stage + (size_t)st * selems + t;
            const float4* xt = stage + (size_t)st * selems + belems;
            float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
#pragma unroll
            for (int kk = 0; kk < KPT; ++kk) {
                int b = s + 4 * kk;
                if (b < q2) {
                    float4 kv = Kb[kk * stride];
                    float4 x = xt[b];
                    // (Kr + i Ki)(xr + i xi) = (Kr xr - Ki xi) + i (Kr xi + Ki xr)
                    df_mac(kv.x, kv.y, x.x, x.y, rh, rl);
                    df_mac(-kv.z, -kv.w, x.z, x.w, rh, rl);
                    df_mac(kv.x, kv.y, x.z, x.w, ih, il);
                    df_mac(kv.z, kv.w, x.x, x.y, ih, il);
                }
            }
            accr += (double)rh + (double)rl;
            acci += (double)ih + (double)il;
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (t == 0 && i + NST < n) {
            float4* dst = stage + (size_t)st * selems;
            hmbar_expect_tx(&full[st], kbytes + xbytes);
            hbulk_load(dst, K + (b0 + i + NST) * (int64_t)belems, kbytes, &full[st]);
            hbulk_load(dst + belems, xr + (int64_t)srcs[i + NST] * q2p, xbytes, &full[st]);
        }
    }
    if (failed) {
        if (t == 0) {
            atomicOr(status, 1);
            for (int j = i; j < n && j < i + NST; ++j) hmbar_wait(&full[j % NST], (unsigned)((j / NST) & 1), 1LL << 24);
        }
        __syncthreads();
        return;
    }
    accr += __shfl_xor_sync(0xffffffffu, accr, 1);
    accr += __shfl_xor_sync(0xffffffffu, accr, 2);
    acci += __shfl_xor_sync(0xffffffffu, acci, 1);
    acci += __shfl_xor_sync(0xffffffffu, acci, 2);
    if (active && s == 0) {
        yh[((2 * r) * C + sigma) * q2 + a] = accr;
        yh[((2 * r + 1) * C + sigma) * q2 + a] = acci;
    }
}

// Complex coupling generated on the fly in FP64 (when the stored matrices would
// not fit): thread (g, a) handles target point a against blocks g, g + G, ...
__global__ void helm_coupling64_otf_kernel(const int32_t* __restrict__ rows, const int64_t* __restrict__ fptr,
                                           const int32_t* __restrict__ fsrc, const double* __restrict__ igeo, int q2,
                                           int G, int R, int64_t C, double kappa, const double* __restrict__ xh,
                                           double* __restrict__ yh) {
    extern __shared__ double red[];
    const int sigma = rows[blockIdx.x];
    const int64_t r = blockIdx.y;
    const int t = threadIdx.x, g = t / q2, a = t % q2;
    double accr = 0.0, acci = 0.0;
    if (g < G) {
        const double* X = igeo + 4 * ((int64_t)sigma * q2 + a);
        const double* xre = xh + (2 * r) * C * q2;
        const double* xim = xh + (2 * r + 1) * C * q2;
        for (int64_t blk = fptr[sigma] + g; blk < fptr[sigma + 1]; blk += G) {
            int64_t tau = fsrc[blk];
            for (int b = 0; b < q2; ++b) {
                const double* Y = igeo + 4 * (tau * q2 + b);
                double d0 = X[0] - Y[0], d1 = X[1] - Y[1], d2 = X[2] - Y[2];
                double kr, ki;
                helm_kernel64(kappa, sqrt(d0 * d0 + d1 * d1 + d2 * d2), X[3] * Y[3], &kr, &ki);
                double vr = xre[tau * q2 + b], vi = xim[tau * q2 + b];
                accr += kr * vr - ki * vi;
                acci += kr * vi + ki * vr;
            }
        }
    }
    red[2 * t] = accr;
    red[2 * t + 1] = acci;
    __syncthreads();
    if (t < q2) {
        double vr = 0.0, vi = 0.0;
        for (int k = 0; k < G; ++k) {
            vr += red[2 * (k * q2 + t)];
            vi += red[2 * (k * q2 + t) + 1];
        }
        yh[((2 * r) * C + sigma) * q2 + t] = vr;
        yh[((2 * r + 1) * C + sigma) * q2 + t] = vi;
    }
}

// Complex coupling generated on the fly in FP32: phase kappa r reduced to
// [-pi, pi] in FP32 before the hardware sine / cosine; the per-block sums are
// accumulated in double.  src32c[t][b] = (x, y, z, k_b / (4 pi)), the moments are
// read as (re, im) floats.
__global__ void helm_coupling32_kernel(const int32_t* __restrict__ rows, const int64_t* __restrict__ fptr,
                                       const int32_t* __restrict__ fsrc, const float* __restrict__ igeo32, int q2,
                                       int G, int64_t C, float kappa, const float2* __restrict__ xh32,
                                       double* __restrict__ yh_re, double* __restrict__ yh_im) {
    extern __shared__ double red[];
    const int sigma = rows[blockIdx.x];
    const int t = threadIdx.x, g = t / q2, a = t % q2;
    double accr = 0.0, acci = 0.0;
    const float inv2pi = 0.15915494309189535f, twopi = 6.283185307179586f;
    if (g < G) {
        const float* X = igeo32 + 4 * ((int64_t)sigma * q2 + a);
        const float x0 = X[0], x1 = X[1], x2 = X[2];
        for (int64_t blk = fptr[sigma] + g; blk < fptr[sigma + 1]; blk += G) {
            const int64_t tau = fsrc[blk];
            const float4* Y = reinterpret_cast<const float4*>(igeo32) + tau * q2;
            const float2* V = xh32 + tau * q2;
            float fr = 0.f, fi = 0.f;
            for (int b = 0; b < q2; ++b) {
                float4 y = Y[b];
                float2 v = V[b];
                float d0 = x0 - y.x, d1 = x1 - y.y, d2 = x2 - y.z;
                float r2 = d0 * d0 + d1 * d1 + d2 * d2;
                float rinv = rsqrtf(r2);
                float ph = kappa * (r2 * rinv);
                ph = fmaf(-twopi, rintf(ph * inv2pi), ph);
                float sn, cs;
                __sincosf(ph, &sn, &cs);
                float w = y.w * rinv;
                float kr = w * cs, ki = w * sn;
                fr = fmaf(kr, v.x, fmaf(-ki, v.y, fr));
                fi = fmaf(kr, v.y, fmaf(ki, v.x, fi));
            }
            accr += (double)fr;
            acci += (double)fi;
        }
    }
    red[2 * t] = accr;
    red[2 * t + 1] = acci;
    __syncthreads();
    if (t < q2) {
        double vr = 0.0, vi = 0.0;
        for (int k = 0; k < G; ++k) {
            vr += red[2 * (k * q2 + t)];
            vi += red[2 * (k * q2 + t) + 1];
        }
        double ka = (double)igeo32[4 * ((int64_t)sigma * q2 + t) + 3] / (4.0 * IBEM_PI);
        yh_re[(int64_t)sigma * q2 + t] = vr * ka;
        yh_im[(int64_t)sigma * q2 + t] = vi * ka;
    }
}

__global__ void helm_src32_kernel(int64_t n, const double* __restrict__ xre, const double* __restrict__ xim,
                                  float2* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2((float)xre[i], (float)xim[i]);
}

// ---- near product (complex) -------------------------------------------------------
// y*_e += sum B x*_s over the row; x*, y* in the split layout (2R real vectors).
template <typename T2, typename T>
__global__ void helm_near_apply_kernel(const int64_t* __restrict__ nptr, const int32_t* __restrict__ nsrc,
                                       const T2* __restrict__ blocks, int nb, int64_t E, const T* __restrict__ xs,
                                       double* __restrict__ ys) {
    extern __shared__ double red[];
    const int64_t e = blockIdx.x, r = blockIdx.y;
    const int t = threadIdx.x, nbb = nb * nb;
    double accr = 0.0, acci = 0.0;
    if (t < nbb) {
        int j = t % nb;
        const T* xre = xs + (2 * r) * E * nb;
        const T* xim = xs + (2 * r + 1) * E * nb;
        T pr = (T)0, pi = (T)0;
        for (int64_t k = nptr[e]; k < nptr[e + 1]; ++k) {
            T2 b = blocks[k * nbb + t];
            int64_t o = (int64_t)nsrc[k] * nb + j;
            T vr = xre[o], vi = xim[o];
            pr += b.x * vr - b.y * vi;
            pi += b.x * vi + b.y * vr;
        }
        accr = (double)pr;
        acci = (double)pi;
    }
    red[2 * t] = accr;
    red[2 * t + 1] = acci;
    __syncthreads();
    if (t < nb) {
        double vr = 0.0, vi = 0.0;
        for (int j = 0; j < nb; ++j) {
            vr += red[2 * (t * nb + j)];
            vi += red[2 * (t * nb + j) + 1];
        }
        ys[((2 * r) * E + e) * nb + t] += vr;
        ys[((2 * r + 1) * E + e) * nb + t] += vi;
    }
}

// FP64-accurate near product for several right-hand sides in double-float on
// the FP32 pipe: one CTA per target element; per near block of its row the
// block (FP64, split into hi + lo pairs) and the source element's lifted
// coefficients of every right-hand side are staged in shared memory, and thread
// (row i, right-hand side r) accumulates sum_j B[i][j] x*_s[j][r] with exact
// products and TwoSum accumulation (as the coupling's double-float arithmetic);
// each block is read once for all right-hand sides.  Adds to ys (split layout).
constexpr int HN_T = 256;

__device__ __forceinline__ void hn_split(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}
__device__ __forceinline__ void hn_mac(float ah, float al, float bh, float bl, float& hi, float& lo) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, fmaf(al, bh, e));
    const float t = hi + p;
    const float z = t - hi;
    const float err = (hi - (t - z)) + (p - z);
    hi = t;
    lo += err + e;
}

__global__ void __launch_bounds__(HN_T) helm_near_df_kernel(const int64_t* __restrict__ nptr,
                                                            const int32_t* __restrict__ nsrc,
                                                            const double2* __restrict__ blocks, int nb, int R,
                                                            int64_t E, const double* __restrict__ xs,
                                                            double* __restrict__ ys) {
    extern __shared__ float4 hn_sm[];
    float4* Bs = hn_sm;              // [nb * nb] (re_h, re_l, im_h, im_l)
    float4* Xs = hn_sm + nb * nb;    // [nb][R]  (re_h, re_l, im_h, im_l)
    const int64_t e = blockIdx.x;
    const int t = threadIdx.x, nbb = nb * nb, np = nb * R;
    constexpr int MAXP = 8;          // (row, right-hand side) pairs per thread: nb R <= 8 HN_T
    float acc[MAXP][4];
#pragma unroll
    for (int k = 0; k < MAXP; ++k) acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = 0.0f;
    for (int64_t k = nptr[e]; k < nptr[e + 1]; ++k) {
        const int64_t s = nsrc[k];
        __syncthreads();   // the previous block is consumed
        for (int q = t; q < nbb; q += HN_T) {
            const double2 b = blocks[k * nbb + q];
            float4 v;
            hn_split(b.x, v.x, v.y);
            hn_split(b.y, v.z, v.w);
            Bs[q] = v;
        }
        for (int q = t; q < np; q += HN_T) {
            const int j = q / R, r = q % R;
            float4 v;
            hn_split(xs[((int64_t)(2 * r) * E + s) * nb + j], v.x, v.y);
            hn_split(xs[((int64_t)(2 * r + 1) * E + s) * nb + j], v.z, v.w);
            Xs[q] = v;
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < MAXP; ++m) {
            const int p = t + HN_T * m;
            if (p < np) {
                const int i = p / R, r = p % R;
                for (int j = 0; j < nb; ++j) {
                    const float4 b = Bs[i * nb + j], x = Xs[j * R + r];
                    // (Br + i Bi)(xr + i xi) = (Br xr - Bi xi) + i (Br xi + Bi xr)
                    hn_mac(b.x, b.y, x.x, x.y, acc[m][0], acc[m][1]);
                    hn_mac(-b.z, -b.w, x.z, x.w, acc[m][0], acc[m][1]);
                    hn_mac(b.x, b.y, x.z, x.w, acc[m][2], acc[m][3]);
                    hn_mac(b.z, b.w, x.x, x.y, acc[m][2], acc[m][3]);
                }
            }
        }
    }
#pragma unroll
    for (int m = 0; m < MAXP; ++m) {
        const int p = t + HN_T * m;
        if (p < np) {
            const int i = p / R, r = p % R;
            ys[((int64_t)(2 * r) * E + e) * nb + i] += (double)acc[m][0] + (double)acc[m][1];
            ys[((int64_t)(2 * r + 1) * E + e) * nb + i] += (double)acc[m][2] + (double)acc[m][3];
        }
    }
}

// ---- layout conversion ---------------------------------------------------------------
// interleaved [R][n][2] <-> split [2R][n]
__global__ void helm_split_vec_kernel(int R, int64_t n, const double* __restrict__ in, double* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)R * n) return;
    int64_t r = i / n, k = i % n;
    out[(2 * r) * n + k] = in[2 * i];
    out[(2 * r + 1) * n + k] = in[2 * i + 1];
}

__global__ void helm_join_vec_kernel(int R, int64_t n, const double* __restrict__ in, double* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)R * n) return;
    int64_t r = i / n, k = i % n;
    out[2 * i] = in[(2 * r) * n + k];
    out[2 * i + 1] = in[(2 * r + 1) * n + k];
}

// ---- potential (complex) -------------------------------------------------------------
// u(x) = sum over Gauss points of W mu exp(i kappa |x - y|) / (4 pi |x - y|);
// srcs[g] = (x, y, z, W mu_re / 4pi), mu_im in srci[g].
// Densities of up to HP_RC right-hand sides at once: mu[s][j] = w_s k_s (mu_re, mu_im) / (4 pi)
// for slot j; positions are written once (pos[s] = (x, y, z, 0)).
constexpr int HP_RC = 16;

__global__ void helm_density_slot_kernel(int64_t E, int QQ, int nb, const double* __restrict__ qgeo,
                                         const double* __restrict__ phi, const double* __restrict__ wre,
                                         const double* __restrict__ wim, int j, double2* __restrict__ mu,
                                         double4_32a* __restrict__ pos) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= E * QQ) return;
    int64_t e = idx / QQ;
    int q = (int)(idx % QQ);
    double mr = 0.0, mi = 0.0;
    for (int i = 0; i < nb; ++i) {
        mr += phi[q * nb + i] * wre[e * nb + i];
        mi += phi[q * nb + i] * wim[e * nb + i];
    }
    const double* X = qgeo + 4 * idx;
    const double s = X[3] / (4.0 * IBEM_PI);
    mu[idx * HP_RC + j] = make_double2(s * mr, s * mi);
    if (pos) pos[idx] = make_double4_32a(X[0], X[1], X[2], 0.0);
}

// u_j(x) += sum_s e^{i kappa r} / r mu[s][j] for the nc densities of a chunk: the
// complex exponential is evaluated once per (point, source) and applied to all
// of them.  Grid: (points, source splits); atomics combine the splits.
__global__ void helm_potential_multi_kernel(int64_t npts, const double* __restrict__ pts, int64_t nsrc,
                                            const double4_32a* __restrict__ pos, const double2* __restrict__ mu,
                                            int nc, int64_t chunk, double kappa, double* __restrict__ u) {
    int64_t ip = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= npts) return;
    double x0 = pts[3 * ip], x1 = pts[3 * ip + 1], x2 = pts[3 * ip + 2];
    int64_t s0 = blockIdx.y * chunk, s1 = s0 + chunk < nsrc ? s0 + chunk : nsrc;
    double ar[HP_RC], ai[HP_RC];
#pragma unroll
    for (int j = 0; j < HP_RC; ++j) ar[j] = ai[j] = 0.0;
    for (int64_t s = s0; s < s1; ++s) {
        const double4_32a y = pos[s];
        const double d0 = x0 - y.x, d1 = x1 - y.y, d2 = x2 - y.z;
        const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        double sn, cs;
        sincos(kappa * r, &sn, &cs);
        const double ir = 1.0 / r;
        const double gr = cs * ir, gi = sn * ir;
        const double2* m = mu + s * HP_RC;
#pragma unroll
        for (int j = 0; j < HP_RC; ++j) {
            if (j < nc) {
                const double2 v = m[j];
                ar[j] += gr * v.x - gi * v.y;
                ai[j] += gr * v.y + gi * v.x;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < HP_RC; ++j) {
        if (j < nc) {
            atomicAdd(u + (size_t)2 * j * npts + 2 * ip, ar[j]);
            atomicAdd(u + (size_t)2 * j * npts + 2 * ip + 1, ai[j]);
        }
    }
}

// ---- host launchers ----------------------------------------------------------------------
cudaError_t helm_launch_near_assembly(ibem_handle* h) {
    Plan& P = h->P;
    GeomView g{h->d_patches, h->d_knots, h->d_cpw};
    int QQ = P.Q * P.Q, nb = P.nb;
    double kappa = P.prm.kappa;
    cudaError_t e;
    std::vector<double> gx, gw;
    gauss_legendre(P.Q, gx, gw);
    if ((e = cudaMemcpyToSymbolAsync(c_hgx, gx.data(), P.Q * sizeof(double), 0, cudaMemcpyHostToDevice, h->stream))) return e;
    if ((e = cudaMemcpyToSymbolAsync(c_hgw, gw.data(), P.Q * sizeof(double), 0, cudaMemcpyHostToDevice, h->stream))) return e;
    double2* blocks = reinterpret_cast<double2*>(h->d_near);
    for (int cls : {CLS_REGULAR, CLS_SUBDIV}) {
        if (h->n_list[cls] > 0 && near_shared_bytes(P.Q, nb, true, cls == CLS_SUBDIV) > IBEM_MAX_SMEM_BYTES &&
            (e = launch_near_stream(h, cls, true, kappa, h->d_near)))
            return e;
    }
    if ((e = launch_near_graded(h, true, kappa, h->d_near))) return e;
    if (h->n_list[CLS_REGULAR] > 0 && near_shared_bytes(P.Q, nb, true, false) <= IBEM_MAX_SMEM_BYTES) {
        size_t sm = (size_t)(8 * QQ + 2 * QQ * QQ + 2 * QQ * nb) * sizeof(double);
        if ((e = cudaFuncSetAttribute(helm_near_regular_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
        helm_near_regular_kernel<<<(unsigned)h->n_list[CLS_REGULAR], 128, sm, h->stream>>>(
            h->d_pairs_by_cls[CLS_REGULAR], h->d_near_tgt, h->d_near_src, h->d_qgeo, h->d_phi, QQ, nb, kappa, blocks);
    }
    if (h->n_list[CLS_SUBDIV] > 0 && near_shared_bytes(P.Q, nb, true, true) <= IBEM_MAX_SMEM_BYTES) {
        size_t sm = (size_t)(32 * QQ + 2 * QQ * QQ + 2 * QQ * nb + 2 * nb * nb) * sizeof(double);
        if ((e = cudaFuncSetAttribute(helm_near_subdiv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
        helm_near_subdiv_kernel<<<(unsigned)h->n_list[CLS_SUBDIV], 128, sm, h->stream>>>(
            g, h->d_pairs_by_cls[CLS_SUBDIV], h->d_near_tgt, h->d_near_src, h->d_phi_sub, P.Q, nb, P.ne1, kappa, blocks);
    }
    for (int c = 0; c < 3; ++c) {
        if (h->n_list[c] == 0) continue;
        const int CH = 128;
        size_t sm = (size_t)3 * nb * CH * sizeof(double);
        if ((e = cudaFuncSetAttribute(helm_near_singular_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
        helm_near_singular_kernel<<<(unsigned)h->n_list[c], CH, sm, h->stream>>>(
            g, h->d_pairs_by_cls[c], h->d_near_tgt, h->d_near_src, h->d_near_orient, h->d_rule[c], h->rule_n[c], P.p,
            P.ne1, kappa, blocks);
    }
    if ((e = cudaGetLastError())) return e;
    int64_t nn = P.n_near * nb * nb;
    helm_to_float_kernel<<<nblk(nn, 256), 256, 0, h->stream>>>(blocks, reinterpret_cast<float2*>(h->d_near32), nn);
    helm_near_diag_kernel<<<nblk(P.N, 128), 128, 0, h->stream>>>(P.N, P.p, P.ne1, h->d_near_ptr, h->d_near_src, blocks,
                                                                 h->d_ext, reinterpret_cast<double2*>(h->d_diag));
    return cudaGetLastError();
}

cudaError_t helm_launch_far_assembly(ibem_handle* h) {
    Plan& P = h->P;
    if (P.n_far == 0 || !h->d_Kc) return cudaSuccess;
    int64_t total = P.n_far * (int64_t)h->kpt * 4 * P.q2;
    helm_far_assemble_kernel<<<nblk(total, 256), 256, 0, h->stream>>>(P.n_far, h->d_far_tgt, h->d_far_src, h->d_igeo,
                                                                      P.q2, h->kpt, P.prm.kappa, h->d_Kc);
    return cudaGetLastError();
}

// y = T A T^T x for the complex operator; x, y interleaved [R][N][2].
cudaError_t helm_apply_operator(ibem_handle* h, const double* x, double* y, int nrhs, int precision,
                                double* xsplit, double* ysplit) {
    Plan& P = h->P;
    cudaStream_t st = h->stream;
    const int R = nrhs, R2 = 2 * nrhs;
    const int T = 256;
    cudaError_t e;
    {
        PhaseTimer pt(h, 0);
        helm_split_vec_kernel<<<nblk((int64_t)R * P.N, T), T, 0, st>>>(R, P.N, x, xsplit);
        lift_kernel<<<nblk(R2 * P.E * P.nb, T), T, 0, st>>>(R2, P.E, P.p, P.ne1, h->d_ext, xsplit, P.N, h->d_xs);
        h->launches += 2;
    }
    if (P.q > 0) {
        const int q2 = P.q2;
        const int64_t leaf_off = P.level_off[P.m];
        PhaseTimer pt1(h, 1);
        leaf_moment_kernel<<<nblk(R2 * P.E * q2, T), T, 0, st>>>(R2, P.E, P.pp, P.q, h->d_M, h->d_xs, leaf_off, P.C,
                                                                  h->d_xh);
        h->launches++;
        for (int L = P.m - 1; L >= 0; --L) {
            int64_t nL = P.level_off[L + 1] - P.level_off[L];
            // separable (S_c applied per direction: 2 q^3 instead of q^4 per child)
            m2m_sep_kernel<<<dim3((unsigned)nL, (unsigned)R2), 64, 0, st>>>(nL, P.level_off[L], P.level_off[L + 1],
                                                                            P.q, h->d_S, P.C, h->d_xh);
            h->launches++;
        }
        if ((e = cudaMemsetAsync(h->d_yh, 0, (size_t)R2 * P.C * q2 * sizeof(double), st))) return e;
        pt1.stop();
        unsigned nrows = (unsigned)h->far_rows.size();
        if (nrows > 0) {
            PhaseTimer pt2(h, 2);
            if (precision == IBEM_FP32) {
                int G = 256 / q2 > 0 ? 256 / q2 : 1;
                int threads = ((G * q2 + 31) / 32) * 32;
                for (int r = 0; r < R; ++r) {
                    helm_src32_kernel<<<nblk(P.C * q2, T), T, 0, st>>>(P.C * q2, h->d_xh + (size_t)(2 * r) * P.C * q2,
                                                                       h->d_xh + (size_t)(2 * r + 1) * P.C * q2,
                                                                       reinterpret_cast<float2*>(h->d_src32));
                    helm_coupling32_kernel<<<nrows, threads, (size_t)2 * threads * sizeof(double), st>>>(
                        h->d_far_rows, h->d_far_ptr, h->d_far_src, h->d_igeo32, q2, G, P.C, (float)P.prm.kappa,
                        reinterpret_cast<const float2*>(h->d_src32), h->d_yh + (size_t)(2 * r) * P.C * q2,
                        h->d_yh + (size_t)(2 * r + 1) * P.C * q2);
                    h->launches += 2;
                }
            } else if (h->d_Kc) {
                const int q2p = (q2 + 1) & ~1;
                helm_split_kernel<<<nblk((int64_t)R * P.C * q2p, T), T, 0, st>>>(R, P.C, q2, q2p, h->d_xh, h->d_xh4);
                int threads = ((4 * q2 + 31) / 32) * 32;
                dim3 grid(nrows, R);
                const size_t sbytes = ((size_t)h->kpt * 4 * q2 + q2p) * sizeof(float4);
                const size_t head = 128 + (((size_t)h->max_far_row * 4 + 15) / 16) * 16;
#define IBEM_HDF_LAUNCH(K_, N_)                                                                                   \
    {                                                                                                             \
        size_t sm = head + (size_t)(N_)*sbytes;                                                                   \
        if ((e = cudaFuncSetAttribute(helm_coupling_df_kernel<K_, N_>,                                           \
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))                     \
            return e;                                                                                             \
        helm_coupling_df_kernel<K_, N_><<<grid, threads, sm, st>>>(h->d_far_rows, h->d_far_ptr, h->d_far_src,    \
                                                                   h->d_Kc, q2, q2p, h->max_far_row, P.C,         \
                                                                   h->d_xh4, h->d_yh, h->wait_limit, h->d_status); \
    }                                                                                                             \
    break;
                switch (h->kpt) {
                    case 1: IBEM_HDF_LAUNCH(1, 8)
                    case 3: IBEM_HDF_LAUNCH(3, 6)
                    case 4: IBEM_HDF_LAUNCH(4, 4)
                    case 7: IBEM_HDF_LAUNCH(7, 3)
                    case 9: IBEM_HDF_LAUNCH(9, 2)
                    case 13: IBEM_HDF_LAUNCH(13, 2)
                    case 16: IBEM_HDF_LAUNCH(16, 2)
                    case 21: IBEM_HDF_LAUNCH(21, 1)
                    case 25: IBEM_HDF_LAUNCH(25, 1)
                    default: return cudaErrorInvalidValue;
                }
#undef IBEM_HDF_LAUNCH
                h->launches += 2;
            } else if (P.prm.fp64_coupling == IBEM_COUPLING_SLICED && sliced_supported(h)) {
                if ((e = launch_coupling_sliced(h, R))) return e;
            } else if (P.prm.fp64_coupling != IBEM_COUPLING_NATIVE && gen_supported(h)) {
                if ((e = launch_coupling_gen(h, R))) return e;
            } else {
                int G = 256 / q2 > 0 ? 256 / q2 : 1;
                int threads = ((G * q2 + 31) / 32) * 32;
                helm_coupling64_otf_kernel<<<dim3(nrows, R), threads, (size_t)2 * threads * sizeof(double), st>>>(
                    h->d_far_rows, h->d_far_ptr, h->d_far_src, h->d_igeo, q2, G, R, P.C, P.prm.kappa, h->d_xh,
                    h->d_yh);
                h->launches++;
            }
        }
        PhaseTimer pt3(h, 3);
        for (int L = 0; L < P.m; ++L) {
            const int64_t nL = P.level_off[L + 1] - P.level_off[L];
            l2l_sep_kernel<<<dim3((unsigned)nL, (unsigned)R2), 64, 0, st>>>(nL, P.level_off[L], P.level_off[L + 1],
                                                                            P.q, h->d_S, P.C, h->d_yh);
            h->launches++;
        }
        leaf_back_kernel<<<nblk(R2 * P.E * P.nb, T), T, 0, st>>>(R2, P.E, P.pp, P.q, h->d_M, h->d_yh, leaf_off, P.C,
                                                                  h->d_ys);
        h->launches++;
    } else {
        if ((e = cudaMemsetAsync(h->d_ys, 0, (size_t)R2 * P.Nstar * sizeof(double), st))) return e;
    }
    int threads = ((P.nb * P.nb + 31) / 32) * 32;
    PhaseTimer pt4(h, 4);
    if (precision == IBEM_FP32) {
        d2f_kernel<<<nblk(R2 * P.Nstar, T), T, 0, st>>>(h->d_xs, h->d_xs32, R2 * P.Nstar);
        helm_near_apply_kernel<float2, float><<<dim3((unsigned)P.E, R), threads, 2 * threads * sizeof(double), st>>>(
            h->d_near_ptr, h->d_near_src, reinterpret_cast<const float2*>(h->d_near32), P.nb, P.E, h->d_xs32, h->d_ys);
        h->launches += 2;
    } else {
        if (R >= 4 && P.nb * R <= 8 * HN_T) {
            const size_t sm = (size_t)(P.nb * P.nb + P.nb * R) * sizeof(float4);
            if ((e = cudaFuncSetAttribute(helm_near_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
                return e;
            helm_near_df_kernel<<<(unsigned)P.E, HN_T, sm, st>>>(h->d_near_ptr, h->d_near_src,
                                                                 reinterpret_cast<const double2*>(h->d_near), P.nb,
                                                                 R, P.E, h->d_xs, h->d_ys);
        } else {
            helm_near_apply_kernel<double2, double><<<dim3((unsigned)P.E, R), threads, 2 * threads * sizeof(double),
                                                      st>>>(h->d_near_ptr, h->d_near_src,
                                                            reinterpret_cast<const double2*>(h->d_near), P.nb, P.E,
                                                            h->d_xs, h->d_ys);
        }
        h->launches++;
    }
    pt4.stop();
    PhaseTimer pt5(h, 5);
    restrict_kernel<<<nblk(R2 * P.N, T), T, 0, st>>>(R2, P.N, P.p, P.ne1, h->d_ext, h->d_ys, P.E, ysplit);
    helm_join_vec_kernel<<<nblk((int64_t)R * P.N, T), T, 0, st>>>(R, P.N, ysplit, y);
    h->launches += 2;
    return cudaGetLastError();
}

cudaError_t helm_launch_rhs(ibem_handle* h, const double* g, int nrhs, double* b, double* gsplit, double* bsplit) {
    Plan& P = h->P;
    const int T = 256, R2 = 2 * nrhs;
    int QQ = P.Q * P.Q;
    helm_split_vec_kernel<<<nblk((int64_t)nrhs * P.nq, T), T, 0, h->stream>>>(nrhs, P.nq, g, gsplit);
    rhs_super_kernel<<<nblk(R2 * P.E * P.nb, T), T, 0, h->stream>>>(R2, P.E, QQ, P.nb, h->d_qgeo, h->d_phi, gsplit,
                                                                     P.nq, h->d_ys);
    restrict_kernel<<<nblk(R2 * P.N, T), T, 0, h->stream>>>(R2, P.N, P.p, P.ne1, h->d_ext, h->d_ys, P.E, bsplit);
    helm_join_vec_kernel<<<nblk((int64_t)nrhs * P.N, T), T, 0, h->stream>>>(nrhs, P.N, bsplit, b);
    return cudaGetLastError();
}

cudaError_t helm_launch_potential(ibem_handle* h, const double* w, int nrhs, const double* pts, int64_t npts,
                                  double* u, double* wsplit) {
    Plan& P = h->P;
    cudaError_t e;
    const int T = 256;
    int QQ = P.Q * P.Q;
    int64_t nsrc = P.E * QQ;
    double4_32a* pos = nullptr;
    double2* mu = nullptr;
    if ((e = cudaMallocAsync(&pos, (size_t)nsrc * sizeof(double4_32a), h->stream))) return e;
    if ((e = cudaMallocAsync(&mu, (size_t)nsrc * HP_RC * sizeof(double2), h->stream))) {
        cudaFreeAsync(pos, h->stream);
        return e;
    }
    if ((e = cudaMemsetAsync(u, 0, (size_t)2 * nrhs * npts * sizeof(double), h->stream))) return e;
    int64_t nsplit = (608 * 128) / (npts > 0 ? npts : 1);
    if (nsplit < 1) nsplit = 1;
    if (nsplit > 65535) nsplit = 65535;
    int64_t chunk = (nsrc + nsplit - 1) / nsplit;
    nsplit = (nsrc + chunk - 1) / chunk;
    helm_split_vec_kernel<<<nblk((int64_t)nrhs * P.N, T), T, 0, h->stream>>>(nrhs, P.N, w, wsplit);
    for (int r0 = 0; r0 < nrhs && npts > 0; r0 += HP_RC) {
        const int nc = nrhs - r0 < HP_RC ? nrhs - r0 : HP_RC;
        for (int j = 0; j < nc; ++j) {
            lift_kernel<<<nblk(2 * P.E * P.nb, T), T, 0, h->stream>>>(2, P.E, P.p, P.ne1, h->d_ext,
                                                                      wsplit + (size_t)2 * (r0 + j) * P.N, P.N,
                                                                      h->d_xs);
            helm_density_slot_kernel<<<nblk(nsrc, T), T, 0, h->stream>>>(
                P.E, QQ, P.nb, h->d_qgeo, h->d_phi, h->d_xs, h->d_xs + P.Nstar, j, mu,
                (r0 == 0 && j == 0) ? pos : nullptr);
        }
        helm_potential_multi_kernel<<<dim3(nblk(npts, 128), (unsigned)nsplit), 128, 0, h->stream>>>(
            npts, pts, nsrc, pos, mu, nc, chunk, P.prm.kappa, u + (size_t)2 * r0 * npts);
    }
    cudaError_t le = cudaGetLastError();
    cudaFreeAsync(pos, h->stream);
    cudaFreeAsync(mu, h->stream);
    return le;
}

}  // namespace ibem
