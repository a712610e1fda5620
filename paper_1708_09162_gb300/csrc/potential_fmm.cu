// Potential evaluation with the interpolated far field.
//
// The representation formula (Eq. repform) u(x) = int_Gamma u*(x, y) w(y) dy is
// split per evaluation point over the cluster tree (Sec. 4.1): on a cluster tau
// that is admissible for x (the point taken as a ball of radius 0 in Def. 4.1:
// eta * diam(tau) < max(0, |x - c_tau| - r_tau)) the integrand u*(x, F(y)) k(y)
// is replaced by its tensor Chebyshev interpolant (Sec. 4.2), so that
//     int_tau u*(x, F(y)) k(y) w(y) dy  ~  sum_b u*(x, F(z_b)) k(z_b) x^_tau[b],
// with x^_tau[b] = int_tau L_b^tau w the forward moments of the density.
// Non-admissible elements are summed with the regular Gauss rule of the direct
// evaluation.
//
// Steps: (1) per point, a depth-first walk of the tree counts its far clusters
// and near elements and marks the clusters it uses (one host round trip sizes
// the lists and numbers the marked clusters); (2) the walk again, writing the
// lists; (3) the moments of the marked clusters only, by projecting the
// B-spline coefficients of each density onto the cluster's Lagrange basis one
// direction at a time, x^ = mu_v^T X mu_u with the 1D tables
// mu[j][a] = int L_a b_j over the cluster's interval (the points of a typical
// evaluation use few, coarse clusters, so this is far cheaper than the leaf
// moments and M2M transfers of every cluster); (4) one CTA per (point, chunk
// of PF_RC densities) sums the far and near terms and reduces them in a fixed
// order, so repeated calls give identical results.
#include <algorithm>
#include <vector>

#include "ibem_internal.cuh"

namespace ibem {

namespace {

constexpr int PF_STACK = 32;   // depth-first stack below one root: at most 3 m + 1 <= 31 entries (m <= 10)
constexpr int PF_RC = 16;      // densities per CTA of the evaluation
constexpr int PF_MV = 8;       // real vectors per CTA of the cluster moments
constexpr int PF_T = 256;

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

struct LevelOffsets {
    int64_t off[12];           // cluster id of (level l, patch, morton) = off[l] + patch 4^l + morton
};

// One thread per point.  fill == false: cnt[2 i] = far clusters, cnt[2 i + 1] =
// near elements, used[c] = 1 for every far cluster.  fill == true: writes the
// lists at far_off[i], near_off[i].
__global__ void pf_lists_kernel(int64_t npts, const double* __restrict__ pts, int npatch, int m, LevelOffsets lo,
                                const double* __restrict__ balls, double eta, bool fill, int32_t* __restrict__ cnt,
                                uint8_t* __restrict__ used, const int64_t* __restrict__ far_off,
                                const int64_t* __restrict__ near_off, int32_t* __restrict__ far_list,
                                int32_t* __restrict__ near_list, int* __restrict__ status) {
    const int64_t ip = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= npts) return;
    const double x0 = pts[3 * ip], x1 = pts[3 * ip + 1], x2 = pts[3 * ip + 2];
    int32_t sid[PF_STACK];
    int8_t slv[PF_STACK];
    int64_t nf = 0, nn = 0;
    const int64_t fo = fill ? far_off[ip] : 0, no = fill ? near_off[ip] : 0;
    for (int patch = 0; patch < npatch; ++patch) {
        int sp = 0;
        sid[sp] = (int32_t)(lo.off[0] + patch);
        slv[sp++] = 0;
        while (sp > 0) {
            --sp;
            const int32_t c = sid[sp];
            const int l = slv[sp];
            const double* b = balls + 4 * (int64_t)c;
            const double d0 = x0 - b[0], d1 = x1 - b[1], d2 = x2 - b[2];
            double dist = sqrt(d0 * d0 + d1 * d1 + d2 * d2) - b[3];
            if (!(dist > 0.0)) dist = 0.0;
            if (eta * 2.0 * b[3] < dist) {
                if (fill) far_list[fo + nf] = c;
                else used[c] = 1;
                ++nf;
            } else if (l == m) {
                if (fill) near_list[no + nn] = (int32_t)(c - lo.off[m]);
                ++nn;
            } else {
                if (sp + 4 > PF_STACK) {   // unreachable for m <= 10; recorded, never overrun
                    atomicOr(status, IBEM_DEVICE_OVERFLOW);
                    return;
                }
                const int64_t first = lo.off[l + 1] + 4 * (c - lo.off[l]);
                for (int k = 0; k < 4; ++k) {
                    sid[sp] = (int32_t)(first + k);
                    slv[sp++] = (int8_t)(l + 1);
                }
            }
        }
    }
    if (!fill) {
        cnt[2 * ip] = (int32_t)nf;
        cnt[2 * ip + 1] = (int32_t)nn;
    }
}

// Moments of the marked clusters: one CTA per (cluster, chunk of PF_MV real
// vectors).  Cluster tau = (patch, level l, ix, iy) covers s = 2^(m-l) elements
// per direction and the w = s + p B-splines j = ix s .. ix s + w - 1 that meet
// it; mu[l] is [2^l][w][q] (row jj = j - ix s).  T[jv][au] = sum_ju X[jv][ju]
// mu_u[ju][au] in shared memory, then x^[av q + au] = sum_jv mu_v[jv][av] T[jv][au].
__global__ void pf_moments_kernel(int n_used, const int32_t* __restrict__ used_ids, int R2, int m, int p, int q,
                                  int64_t n1, int64_t N, LevelOffsets lo, const int64_t* __restrict__ mu_off,
                                  const double* __restrict__ mu, const double* __restrict__ x,
                                  double* __restrict__ xhat) {
    extern __shared__ double T[];
    const int u = blockIdx.x;
    const int64_t c = used_ids[u];
    int l = 0;
    while (l < m && c >= lo.off[l + 1]) ++l;
    const int64_t rel = c - lo.off[l];
    const int64_t per = (int64_t)1 << (2 * l);
    const int patch = (int)(rel / per);
    uint32_t ix, iy;
    morton2_inv((uint32_t)(rel % per), &ix, &iy);
    const int s = 1 << (m - l), w = s + p, q2 = q * q;
    const double* mu_u = mu + mu_off[l] + (int64_t)ix * w * q;
    const double* mu_v = mu + mu_off[l] + (int64_t)iy * w * q;
    const int r1 = (blockIdx.y + 1) * PF_MV < R2 ? (blockIdx.y + 1) * PF_MV : R2;
    for (int r = blockIdx.y * PF_MV; r < r1; ++r) {
        const double* X = x + r * N + patch * n1 * n1 + (int64_t)iy * s * n1 + (int64_t)ix * s;
        for (int idx = threadIdx.x; idx < w * q; idx += blockDim.x) {
            const int jv = idx / q, au = idx % q;
            const double* row = X + (int64_t)jv * n1;
            double acc = 0.0;
            for (int ju = 0; ju < w; ++ju) acc = fma(row[ju], mu_u[ju * q + au], acc);
            T[idx] = acc;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < q2; idx += blockDim.x) {
            const int av = idx / q, au = idx % q;
            double acc = 0.0;
            for (int jv = 0; jv < w; ++jv) acc = fma(mu_v[jv * q + av], T[jv * q + au], acc);
            xhat[((int64_t)r * n_used + u) * q2 + idx] = acc;
        }
        __syncthreads();
    }
}

template <bool CPLX>
__device__ __forceinline__ void pf_kernel_value(double d, double kappa, double* gr, double* gi) {
    const double inv = 1.0 / (4.0 * IBEM_PI * d);
    if constexpr (CPLX) {
        double s, c;
        sincos(kappa * d, &s, &c);
        *gr = c * inv;
        *gi = s * inv;
    } else {
        *gr = inv;
        *gi = 0.0;
    }
}

// One CTA per (point, chunk of PF_RC densities).  Far terms: entries (cluster,
// interpolation point b) of the point's list, flattened over the CTA's
// threads; the moments of R densities (complex: 2 R real vectors, real part
// first) are [R][n_used][q2], cluster c at row slot[c].  Near terms: entries
// (element, Gauss point); the density at a Gauss point is
// sum_i phi[g][i] x*_e[i] from the lifted coefficients xs [R][E][nb].
template <bool CPLX>
__global__ void __launch_bounds__(PF_T) pf_eval_kernel(
    int64_t npts, const double* __restrict__ pts, int R, const int64_t* __restrict__ far_off,
    const int32_t* __restrict__ far_list, const int64_t* __restrict__ near_off, const int32_t* __restrict__ near_list,
    int q2, int64_t n_used, const int32_t* __restrict__ slot, const double* __restrict__ igeo,
    const double* __restrict__ xh, int QQ, int nb, int64_t E,
    const double* __restrict__ qgeo, const double* __restrict__ phi, const double* __restrict__ xs, double kappa,
    double* __restrict__ u) {
    constexpr int NA = CPLX ? 2 * PF_RC : PF_RC;
    __shared__ double red[PF_T / 32][NA];
    const int64_t ip = blockIdx.x;
    const int r0 = blockIdx.y * PF_RC;
    const int nc = R - r0 < PF_RC ? R - r0 : PF_RC;
    const double x0 = pts[3 * ip], x1 = pts[3 * ip + 1], x2 = pts[3 * ip + 2];
    double acc[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) acc[j] = 0.0;
    const int64_t CW = CPLX ? 2 : 1;
    // far field
    const int64_t f0 = far_off[ip], nfe = (far_off[ip + 1] - f0) * q2;
    for (int64_t idx = threadIdx.x; idx < nfe; idx += PF_T) {
        const int64_t c = far_list[f0 + idx / q2];
        const int b = (int)(idx % q2);
        const double* z = igeo + 4 * (c * q2 + b);
        const double d0 = x0 - z[0], d1 = x1 - z[1], d2 = x2 - z[2];
        double gr, gi;
        pf_kernel_value<CPLX>(sqrt(d0 * d0 + d1 * d1 + d2 * d2), kappa, &gr, &gi);
        gr *= z[3];
        gi *= z[3];
        const int64_t C = n_used;
        const double* mom = xh + (CW * r0 * C + slot[c]) * q2 + b;
#pragma unroll
        for (int j = 0; j < PF_RC; ++j) {
            if (j < nc) {
                if constexpr (CPLX) {
                    const double mr = mom[(2 * j) * C * q2], mi = mom[(2 * j + 1) * C * q2];
                    acc[2 * j] = fma(gr, mr, fma(-gi, mi, acc[2 * j]));
                    acc[2 * j + 1] = fma(gr, mi, fma(gi, mr, acc[2 * j + 1]));
                } else {
                    acc[j] = fma(gr, mom[j * C * q2], acc[j]);
                }
            }
        }
    }
    // near field
    const int64_t n0 = near_off[ip], nne = (near_off[ip + 1] - n0) * QQ;
    for (int64_t idx = threadIdx.x; idx < nne; idx += PF_T) {
        const int64_t e = near_list[n0 + idx / QQ];
        const int g = (int)(idx % QQ);
        const double* y = qgeo + 4 * (e * QQ + g);
        const double d0 = x0 - y[0], d1 = x1 - y[1], d2 = x2 - y[2];
        double gr, gi;
        pf_kernel_value<CPLX>(sqrt(d0 * d0 + d1 * d1 + d2 * d2), kappa, &gr, &gi);
        gr *= y[3];
        gi *= y[3];
        const double* ph = phi + (int64_t)g * nb;
#pragma unroll
        for (int j = 0; j < PF_RC; ++j) {
            if (j < nc) {
                if constexpr (CPLX) {
                    const double* cr = xs + ((2 * (r0 + j)) * E + e) * nb;
                    const double* ci = xs + ((2 * (r0 + j) + 1) * E + e) * nb;
                    double dr = 0.0, di = 0.0;
                    for (int i = 0; i < nb; ++i) {
                        dr = fma(ph[i], cr[i], dr);
                        di = fma(ph[i], ci[i], di);
                    }
                    acc[2 * j] = fma(gr, dr, fma(-gi, di, acc[2 * j]));
                    acc[2 * j + 1] = fma(gr, di, fma(gi, dr, acc[2 * j + 1]));
                } else {
                    const double* cr = xs + ((int64_t)(r0 + j) * E + e) * nb;
                    double dr = 0.0;
                    for (int i = 0; i < nb; ++i) dr = fma(ph[i], cr[i], dr);
                    acc[j] = fma(gr, dr, acc[j]);
                }
            }
        }
    }
    // fixed-order reduction: butterfly within each warp, then warps in order
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        double v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < NA) {
        const int j = threadIdx.x;
        double s = 0.0;
        for (int w = 0; w < PF_T / 32; ++w) s += red[w][j];
        const int rr = CPLX ? j / 2 : j;
        if (rr < nc) {
            if constexpr (CPLX) u[((int64_t)(r0 + rr) * npts + ip) * 2 + (j & 1)] = s;
            else u[(int64_t)(r0 + rr) * npts + ip] = s;
        }
    }
}

}  // namespace

namespace {

// Temporary device buffers of one call, released on the stream in any case.
struct StreamBuffers {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit StreamBuffers(cudaStream_t s) : st(s) {}
    template <typename T>
    cudaError_t alloc(T** p, size_t n) {
        *p = nullptr;
        cudaError_t e = cudaMallocAsync((void**)p, (n > 0 ? n : 1) * sizeof(T), st);
        if (!e) ptrs.push_back(*p);
        return e;
    }
    ~StreamBuffers() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
};

// 1D moment tables of every level (host, once per handle): for the cluster
// interval i of level l, mu[jj][a] = int L_a(local) b_{i s + jj}, jj < s + p,
// with ceil((q + p) / 2) + 1 Gauss points per element (exact: the integrand is
// a polynomial of degree q - 1 + p on each element).  The B-splines come from
// the handle's Bezier extraction, b_{k + r}(t) = sum_i ext[k][r][i] B_i(t).
cudaError_t ensure_mu1d(ibem_handle* h) {
    if (h->d_mu1d) return cudaSuccess;
    const Plan& P = h->P;
    const int pp = P.pp, q = P.q, ne1 = P.ne1;
    std::vector<double> ext((size_t)ne1 * pp * pp);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(ext.data(), h->d_ext, ext.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream)) ||
        (e = cudaStreamSynchronize(h->stream)))
        return e;
    std::vector<double> z, gx, gw;
    chebyshev_nodes(q, z);
    gauss_legendre((q + P.p + 1) / 2 + 1, gx, gw);
    std::vector<int64_t> off(P.m + 2, 0);
    for (int l = 0; l <= P.m; ++l) off[l + 1] = off[l] + ((int64_t)1 << l) * ((1 << (P.m - l)) + P.p) * q;
    std::vector<double> mu((size_t)off[P.m + 1], 0.0), L(q);
    double B[IBEM_MAX_P + 1];
    const double hel = 1.0 / ne1;
    for (int l = 0; l <= P.m; ++l) {
        const int s = 1 << (P.m - l), w = s + P.p;
        for (int i = 0; i < (1 << l); ++i)
            for (int k = i * s; k < (i + 1) * s; ++k)
                for (size_t g = 0; g < gx.size(); ++g) {
                    lagrange_values(z, ((k - i * s) + gx[g]) / s, L.data());
                    bernstein(P.p, gx[g], B);
                    for (int r = 0; r < pp; ++r) {
                        double bv = 0.0;
                        for (int t = 0; t < pp; ++t) bv += ext[((size_t)k * pp + r) * pp + t] * B[t];
                        double* row = mu.data() + off[l] + ((int64_t)i * w + (k - i * s + r)) * q;
                        for (int a = 0; a < q; ++a) row[a] += gw[g] * hel * bv * L[a];
                    }
                }
    }
    if ((e = cudaMalloc(&h->d_mu1d, mu.size() * sizeof(double))) ||
        (e = cudaMemcpyAsync(h->d_mu1d, mu.data(), mu.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream)) ||
        (e = cudaMalloc(&h->d_mu1d_off, off.size() * sizeof(int64_t))) ||
        (e = cudaMemcpyAsync(h->d_mu1d_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                             h->stream)) ||
        (e = cudaStreamSynchronize(h->stream)))
        return e;
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_potential_fmm(ibem_handle* h, const double* w, int nrhs, const double* pts, int64_t npts,
                                 double* u, int64_t* n_far_terms, int64_t* n_near_terms) {
    Plan& P = h->P;
    cudaStream_t st = h->stream;
    cudaError_t e;
    const int T = 256;
    const int R2 = h->helm ? 2 * nrhs : nrhs;
    if ((e = ensure_mu1d(h))) return e;
    StreamBuffers buf(st);
    // (1) count, mark the clusters used
    LevelOffsets lo{};
    for (int l = 0; l <= P.m + 1 && l < 12; ++l) lo.off[l] = P.level_off[l];
    int32_t* d_cnt;
    uint8_t* d_used;
    if ((e = buf.alloc(&d_cnt, (size_t)2 * npts)) || (e = buf.alloc(&d_used, (size_t)P.C)) ||
        (e = cudaMemsetAsync(d_used, 0, (size_t)P.C, st)))
        return e;
    pf_lists_kernel<<<nblk(npts, 128), 128, 0, st>>>(npts, pts, P.npatch, P.m, lo, h->d_balls, P.prm.eta, false, d_cnt,
                                                      d_used, nullptr, nullptr, nullptr, nullptr, h->d_status);
    h->launches++;
    std::vector<int32_t> cnt((size_t)2 * npts);
    std::vector<uint8_t> used((size_t)P.C);
    if ((e = cudaMemcpyAsync(cnt.data(), d_cnt, cnt.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(used.data(), d_used, used.size(), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
        return e;
    std::vector<int64_t> off((size_t)2 * (npts + 1), 0);   // far offsets, then near offsets
    for (int64_t i = 0; i < npts; ++i) {
        off[i + 1] = off[i] + cnt[2 * i];
        off[npts + 1 + i + 1] = off[npts + 1 + i] + cnt[2 * i + 1];
    }
    const int64_t nfar = off[npts], nnear = off[2 * npts + 1];
    if (n_far_terms) *n_far_terms = nfar;
    if (n_near_terms) *n_near_terms = nnear;
    std::vector<int32_t> ids, slot((size_t)P.C, -1);
    int wmax = 1;
    for (int64_t c = 0; c < P.C; ++c)
        if (used[c]) {
            slot[c] = (int32_t)ids.size();
            ids.push_back((int32_t)c);
            int pa, l, ix, iy;
            cluster_of(P, c, &pa, &l, &ix, &iy);
            wmax = std::max(wmax, (1 << (P.m - l)) + P.p);
        }
    const int n_used = (int)ids.size();
    // (2) lists
    int64_t* d_off;
    int32_t *d_lists, *d_ids, *d_slot;
    if ((e = buf.alloc(&d_off, off.size())) || (e = buf.alloc(&d_lists, (size_t)(nfar + nnear))) ||
        (e = buf.alloc(&d_ids, ids.size())) || (e = buf.alloc(&d_slot, slot.size())) ||
        (e = cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(d_slot, slot.data(), slot.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st)))
        return e;
    if (n_used > 0 && (e = cudaMemcpyAsync(d_ids, ids.data(), ids.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                           st)))
        return e;
    pf_lists_kernel<<<nblk(npts, 128), 128, 0, st>>>(npts, pts, P.npatch, P.m, lo, h->d_balls, P.prm.eta, true, d_cnt,
                                                      nullptr, d_off, d_off + npts + 1, d_lists, d_lists + nfar,
                                                      h->d_status);
    h->launches++;
    // (3) densities as real vectors, moments of the used clusters, lifted
    // coefficients for the near elements
    const double* wr = w;
    if (h->helm) {
        double* d_split;
        if ((e = buf.alloc(&d_split, (size_t)R2 * P.N))) return e;
        helm_split_vec_kernel<<<nblk((int64_t)nrhs * P.N, T), T, 0, st>>>(nrhs, P.N, w, d_split);
        wr = d_split;
        h->launches++;
    }
    double *d_xhat, *d_xs = nullptr;
    if ((e = buf.alloc(&d_xhat, (size_t)R2 * (n_used > 0 ? n_used : 1) * P.q2))) return e;
    if (n_used > 0) {
        const size_t sm = (size_t)wmax * P.q * sizeof(double);
        if ((e = cudaFuncSetAttribute(pf_moments_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
            return e;
        pf_moments_kernel<<<dim3((unsigned)n_used, (unsigned)((R2 + PF_MV - 1) / PF_MV)), 128, sm, st>>>(
            n_used, d_ids, R2, P.m, P.p, P.q, P.n1, P.N, lo, h->d_mu1d_off, h->d_mu1d, wr, d_xhat);
        h->launches++;
    }
    if (nnear > 0) {
        if ((e = buf.alloc(&d_xs, (size_t)R2 * P.Nstar))) return e;
        lift_kernel<<<nblk((int64_t)R2 * P.E * P.nb, T), T, 0, st>>>(R2, P.E, P.p, P.ne1, h->d_ext, wr, P.N, d_xs);
        h->launches++;
    }
    // (4) evaluation
    dim3 grid((unsigned)npts, (unsigned)((nrhs + PF_RC - 1) / PF_RC));
    const int QQ = P.Q * P.Q;
    if (h->helm)
        pf_eval_kernel<true><<<grid, PF_T, 0, st>>>(npts, pts, nrhs, d_off, d_lists, d_off + npts + 1,
                                                    d_lists + nfar, P.q2, n_used, d_slot, h->d_igeo, d_xhat, QQ,
                                                    P.nb, P.E, h->d_qgeo, h->d_phi, d_xs, P.prm.kappa, u);
    else
        pf_eval_kernel<false><<<grid, PF_T, 0, st>>>(npts, pts, nrhs, d_off, d_lists, d_off + npts + 1,
                                                     d_lists + nfar, P.q2, n_used, d_slot, h->d_igeo, d_xhat, QQ,
                                                     P.nb, P.E, h->d_qgeo, h->d_phi, d_xs, 0.0, u);
    h->launches++;
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Right-hand side of a field of point sources with the interpolated far field.
//
// For g(x) = sum_j c_j u*(x, y_j) the Galerkin right-hand side (Sec. 3.2)
// b*_i = int_Gamma g b*_i is the transpose of the interpolated potential (u* is
// symmetric): per source the tree is walked as for a potential point; on a
// cluster sigma admissible for y_j the integrand k(x^) u*(F(x^), y_j) is
// replaced by its interpolant (Sec. 4.2), so the source adds c_j k(z_a)
// u*(F(z_a), y_j) to the value at node a of sigma; elements that are never
// admissible take the regular Gauss rule.  The node values of every cluster
// then run through the operator's own downward pass (separable L2L, leaf
// back-projection with the moments int L_a b*_i) and the restriction T.
// The per-source lists come from pf_lists_kernel; the host transposes them
// into lists per cluster and per element with the sources ascending, so every
// sum runs in a fixed order and repeated calls give identical results.
namespace {

constexpr int RS_T = 256;    // threads per CTA of the right-hand-side kernels
constexpr int RS_RC = 8;     // charge vectors per CTA

// Far values: one CTA per (cluster with sources admissible for it, chunk of
// RS_RC charge vectors).  Thread t takes node a = t % q2 and every np-th
// source of the cluster's list (part t / q2, np = RS_T / q2 parts); the parts
// are summed in order.  Output in the split real layout [R2][C][q2].
template <bool CPLX>
__global__ void __launch_bounds__(RS_T) rs_far_kernel(
    const int32_t* __restrict__ clusters, const int64_t* __restrict__ cptr, const int32_t* __restrict__ csrc,
    const double* __restrict__ src, const double* __restrict__ charges, int R, int64_t nsrc, int q2, int64_t C,
    const double* __restrict__ igeo, double kappa, double* __restrict__ yh) {
    constexpr int CW = CPLX ? 2 : 1;
    constexpr int NV = RS_RC * CW;
    __shared__ double part[NV * RS_T];
    const int u = blockIdx.x;
    const int64_t c = clusters[u];
    const int r0 = blockIdx.y * RS_RC;
    const int nc = R - r0 < RS_RC ? R - r0 : RS_RC;
    const int np = RS_T / q2;
    const int t = threadIdx.x, a = t % q2, pp = t / q2;
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    if (pp < np) {
        const double* z = igeo + 4 * (c * q2 + a);
        const double z0 = z[0], z1 = z[1], z2 = z[2];
        for (int64_t k = cptr[u] + pp; k < cptr[u + 1]; k += np) {
            const int64_t j = csrc[k];
            const double d0 = z0 - src[3 * j], d1 = z1 - src[3 * j + 1], d2 = z2 - src[3 * j + 2];
            double gr, gi;
            pf_kernel_value<CPLX>(sqrt(d0 * d0 + d1 * d1 + d2 * d2), kappa, &gr, &gi);
#pragma unroll
            for (int rr = 0; rr < RS_RC; ++rr) {
                if (rr < nc) {
                    if constexpr (CPLX) {
                        const double* qc = charges + ((int64_t)(r0 + rr) * nsrc + j) * 2;
                        const double qr = qc[0], qi = qc[1];
                        acc[2 * rr] = fma(gr, qr, fma(-gi, qi, acc[2 * rr]));
                        acc[2 * rr + 1] = fma(gr, qi, fma(gi, qr, acc[2 * rr + 1]));
                    } else {
                        acc[rr] = fma(gr, charges[(int64_t)(r0 + rr) * nsrc + j], acc[rr]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) part[v * RS_T + t] = acc[v];
    __syncthreads();
    if (t < q2) {
        const double kz = igeo[4 * (c * q2 + t) + 3];
        for (int v = 0; v < nc * CW; ++v) {
            double sum = 0.0;
            for (int k = 0; k < np; ++k) sum += part[v * RS_T + k * q2 + t];
            const int rr = v / CW, comp = v % CW;
            const int64_t vec = CPLX ? 2 * (int64_t)(r0 + rr) + comp : (int64_t)(r0 + rr);
            yh[(vec * C + c) * q2 + t] = sum * kz;
        }
    }
}

// Near sums: one CTA per (element with near sources, chunk of RS_RC charge
// vectors).  Gauss points in chunks of RS_T: each thread forms W_g g(x_g) at
// its point from the element's sources (in list order) into shared memory,
// then the (dof, component) entries sum phi[g][i] over the chunk in order.
// Adds to ys [R2][E][nb] (written by the leaf back-projection before).
template <bool CPLX>
__global__ void __launch_bounds__(RS_T) rs_near_kernel(
    const int32_t* __restrict__ elems, const int64_t* __restrict__ eptr, const int32_t* __restrict__ esrc,
    const double* __restrict__ src, const double* __restrict__ charges, int R, int64_t nsrc, int QQ, int nb,
    int64_t E, const double* __restrict__ qgeo, const double* __restrict__ phi, double kappa,
    double* __restrict__ ys) {
    constexpr int CW = CPLX ? 2 : 1;
    constexpr int NV = RS_RC * CW;
    constexpr int MAXO = (25 * NV + RS_T - 1) / RS_T;   // nb <= 25
    __shared__ double sg[NV * RS_T];
    const int64_t e = elems[blockIdx.x];
    const int r0 = blockIdx.y * RS_RC;
    const int nc = R - r0 < RS_RC ? R - r0 : RS_RC;
    const int nout = nb * NV;
    double out[MAXO];
#pragma unroll
    for (int o = 0; o < MAXO; ++o) out[o] = 0.0;
    for (int g0 = 0; g0 < QQ; g0 += RS_T) {
        const int g = g0 + threadIdx.x;
        double val[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) val[v] = 0.0;
        if (g < QQ) {
            const double* x = qgeo + 4 * (e * QQ + g);
            const double x0 = x[0], x1 = x[1], x2 = x[2], w = x[3];
            for (int64_t k = eptr[blockIdx.x]; k < eptr[blockIdx.x + 1]; ++k) {
                const int64_t j = esrc[k];
                const double d0 = x0 - src[3 * j], d1 = x1 - src[3 * j + 1], d2 = x2 - src[3 * j + 2];
                double gr, gi;
                pf_kernel_value<CPLX>(sqrt(d0 * d0 + d1 * d1 + d2 * d2), kappa, &gr, &gi);
                gr *= w;
                gi *= w;
#pragma unroll
                for (int rr = 0; rr < RS_RC; ++rr) {
                    if (rr < nc) {
                        if constexpr (CPLX) {
                            const double* qc = charges + ((int64_t)(r0 + rr) * nsrc + j) * 2;
                            const double qr = qc[0], qi = qc[1];
                            val[2 * rr] = fma(gr, qr, fma(-gi, qi, val[2 * rr]));
                            val[2 * rr + 1] = fma(gr, qi, fma(gi, qr, val[2 * rr + 1]));
                        } else {
                            val[rr] = fma(gr, charges[(int64_t)(r0 + rr) * nsrc + j], val[rr]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) sg[v * RS_T + threadIdx.x] = val[v];
        __syncthreads();
        const int ng = QQ - g0 < RS_T ? QQ - g0 : RS_T;
#pragma unroll
        for (int o = 0; o < MAXO; ++o) {
            const int idx = threadIdx.x + o * RS_T;
            if (idx < nout) {
                const int i = idx / NV, v = idx % NV;
                double sum = 0.0;
                for (int gg = 0; gg < ng; ++gg) sum = fma(phi[(int64_t)(g0 + gg) * nb + i], sg[v * RS_T + gg], sum);
                out[o] += sum;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 0; o < MAXO; ++o) {
        const int idx = threadIdx.x + o * RS_T;
        if (idx < nout) {
            const int i = idx / NV, v = idx % NV, rr = v / CW, comp = v % CW;
            if (rr < nc) {
                const int64_t vec = CPLX ? 2 * (int64_t)(r0 + rr) + comp : (int64_t)(r0 + rr);
                ys[(vec * E + e) * nb + i] += out[o];
            }
        }
    }
}

// Lists per target (cluster or element) from the lists per source: counting
// sort over the sources in order, so each target's sources are ascending.
void transpose_lists(int64_t nsrc, const std::vector<int64_t>& off, const std::vector<int32_t>& lists,
                     int64_t list0, int64_t ntargets, std::vector<int32_t>& targets, std::vector<int64_t>& tptr,
                     std::vector<int32_t>& tsrc) {
    std::vector<int64_t> cnt((size_t)ntargets, 0);
    const int64_t n = off[nsrc] - off[0];
    for (int64_t k = 0; k < n; ++k) cnt[lists[list0 + k]]++;
    std::vector<int64_t> pos((size_t)ntargets, -1);
    targets.clear();
    tptr.assign(1, 0);
    for (int64_t t = 0; t < ntargets; ++t)
        if (cnt[t] > 0) {
            pos[t] = tptr.back();
            targets.push_back((int32_t)t);
            tptr.push_back(tptr.back() + cnt[t]);
        }
    tsrc.assign((size_t)n, 0);
    for (int64_t j = 0; j < nsrc; ++j)
        for (int64_t k = off[j]; k < off[j + 1]; ++k) tsrc[pos[lists[list0 + k - off[0]]]++] = (int32_t)j;
}

}  // namespace

cudaError_t launch_rhs_sources(ibem_handle* h, const double* src, const double* charges, int nrhs, int64_t nsrc,
                               double* b, int64_t* n_far_terms, int64_t* n_near_terms) {
    Plan& P = h->P;
    cudaStream_t st = h->stream;
    cudaError_t e;
    const int T = 256;
    const int R2 = h->helm ? 2 * nrhs : nrhs;
    StreamBuffers buf(st);
    // (1) lists per source (the potential's walk)
    LevelOffsets lo{};
    for (int l = 0; l <= P.m + 1 && l < 12; ++l) lo.off[l] = P.level_off[l];
    int32_t* d_cnt;
    uint8_t* d_used;
    if ((e = buf.alloc(&d_cnt, (size_t)2 * nsrc)) || (e = buf.alloc(&d_used, (size_t)P.C)) ||
        (e = cudaMemsetAsync(d_used, 0, (size_t)P.C, st)))
        return e;
    pf_lists_kernel<<<nblk(nsrc, 128), 128, 0, st>>>(nsrc, src, P.npatch, P.m, lo, h->d_balls, P.prm.eta, false, d_cnt,
                                                      d_used, nullptr, nullptr, nullptr, nullptr, h->d_status);
    h->launches++;
    std::vector<int32_t> cnt((size_t)2 * nsrc);
    if ((e = cudaMemcpyAsync(cnt.data(), d_cnt, cnt.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
        return e;
    std::vector<int64_t> off((size_t)2 * (nsrc + 1), 0);   // far offsets, then near offsets
    for (int64_t i = 0; i < nsrc; ++i) {
        off[i + 1] = off[i] + cnt[2 * i];
        off[nsrc + 1 + i + 1] = off[nsrc + 1 + i] + cnt[2 * i + 1];
    }
    const int64_t nfar = off[nsrc], nnear = off[2 * nsrc + 1];
    if (n_far_terms) *n_far_terms = nfar;
    if (n_near_terms) *n_near_terms = nnear;
    int64_t* d_off;
    int32_t* d_lists;
    if ((e = buf.alloc(&d_off, off.size())) || (e = buf.alloc(&d_lists, (size_t)(nfar + nnear))) ||
        (e = cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st)))
        return e;
    pf_lists_kernel<<<nblk(nsrc, 128), 128, 0, st>>>(nsrc, src, P.npatch, P.m, lo, h->d_balls, P.prm.eta, true, d_cnt,
                                                      nullptr, d_off, d_off + nsrc + 1, d_lists, d_lists + nfar,
                                                      h->d_status);
    h->launches++;
    std::vector<int32_t> lists((size_t)(nfar + nnear));
    if (!lists.empty() &&
        (e = cudaMemcpyAsync(lists.data(), d_lists, lists.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st)))
        return e;
    if ((e = cudaStreamSynchronize(st))) return e;
    // (2) lists per cluster and per element, sources ascending
    std::vector<int64_t> foff(off.begin(), off.begin() + nsrc + 1), noff(off.begin() + nsrc + 1, off.end());
    std::vector<int32_t> cl, csrc, el, esrc;
    std::vector<int64_t> cptr, eptr;
    transpose_lists(nsrc, foff, lists, 0, P.C, cl, cptr, csrc);
    transpose_lists(nsrc, noff, lists, nfar, P.E, el, eptr, esrc);
    int32_t *d_cl = nullptr, *d_csrc = nullptr, *d_el = nullptr, *d_esrc = nullptr;
    int64_t *d_cptr = nullptr, *d_eptr = nullptr;
    auto up32 = [&](int32_t** d, const std::vector<int32_t>& v) -> cudaError_t {
        cudaError_t r = buf.alloc(d, v.size());
        if (r || v.empty()) return r;
        return cudaMemcpyAsync(*d, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    };
    auto up64 = [&](int64_t** d, const std::vector<int64_t>& v) -> cudaError_t {
        cudaError_t r = buf.alloc(d, v.size());
        if (r || v.empty()) return r;
        return cudaMemcpyAsync(*d, v.data(), v.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    };
    if ((e = up32(&d_cl, cl)) || (e = up64(&d_cptr, cptr)) || (e = up32(&d_csrc, csrc)) || (e = up32(&d_el, el)) ||
        (e = up64(&d_eptr, eptr)) || (e = up32(&d_esrc, esrc)))
        return e;
    // (3) node values of the clusters, downward pass, near sums, restriction
    double *d_yh, *d_ys, *d_bs = nullptr;
    if ((e = buf.alloc(&d_yh, (size_t)R2 * P.C * P.q2)) || (e = buf.alloc(&d_ys, (size_t)R2 * P.Nstar)) ||
        (e = cudaMemsetAsync(d_yh, 0, (size_t)R2 * P.C * P.q2 * sizeof(double), st)))
        return e;
    if (h->helm && (e = buf.alloc(&d_bs, (size_t)R2 * P.N))) return e;
    const unsigned nchunk = (unsigned)((nrhs + RS_RC - 1) / RS_RC);
    if (!cl.empty()) {
        dim3 grid((unsigned)cl.size(), nchunk);
        if (h->helm)
            rs_far_kernel<true><<<grid, RS_T, 0, st>>>(d_cl, d_cptr, d_csrc, src, charges, nrhs, nsrc, P.q2, P.C,
                                                       h->d_igeo, P.prm.kappa, d_yh);
        else
            rs_far_kernel<false><<<grid, RS_T, 0, st>>>(d_cl, d_cptr, d_csrc, src, charges, nrhs, nsrc, P.q2, P.C,
                                                        h->d_igeo, 0.0, d_yh);
        h->launches++;
    }
    for (int L = 0; L < P.m; ++L) {
        const int64_t nL = P.level_off[L + 1] - P.level_off[L];
        l2l_sep_kernel<<<dim3((unsigned)nL, (unsigned)R2), 64, 0, st>>>(nL, P.level_off[L], P.level_off[L + 1], P.q,
                                                                       h->d_S, P.C, d_yh);
        h->launches++;
    }
    leaf_back_kernel<<<nblk((int64_t)R2 * P.E * P.nb, T), T, 0, st>>>(R2, P.E, P.pp, P.q, h->d_M, d_yh,
                                                                       P.level_off[P.m], P.C, d_ys);
    h->launches++;
    if (!el.empty()) {
        dim3 grid((unsigned)el.size(), nchunk);
        const int QQ = P.Q * P.Q;
        if (h->helm)
            rs_near_kernel<true><<<grid, RS_T, 0, st>>>(d_el, d_eptr, d_esrc, src, charges, nrhs, nsrc, QQ, P.nb, P.E,
                                                        h->d_qgeo, h->d_phi, P.prm.kappa, d_ys);
        else
            rs_near_kernel<false><<<grid, RS_T, 0, st>>>(d_el, d_eptr, d_esrc, src, charges, nrhs, nsrc, QQ, P.nb,
                                                         P.E, h->d_qgeo, h->d_phi, 0.0, d_ys);
        h->launches++;
    }
    restrict_kernel<<<nblk((int64_t)R2 * P.N, T), T, 0, st>>>(R2, P.N, P.p, P.ne1, h->d_ext, d_ys, P.E,
                                                              h->helm ? d_bs : b);
    h->launches++;
    if (h->helm) {
        helm_join_vec_kernel<<<nblk((int64_t)nrhs * P.N, T), T, 0, st>>>(nrhs, P.N, d_bs, b);
        h->launches++;
    }
    return cudaGetLastError();
}

}  // namespace ibem
