// Lock-step Krylov solver for many right-hand sides (Sec. 4 item 3: conjugate
// gradients for the Laplace single layer, restarted GMRES for Helmholtz; both
// preconditioned by (block) Jacobi).  Every column r of the [R][N] block has its
// own Krylov space, scalars and stopping test, but each step applies the
// operator once to all columns of the block, so the many-right-hand-side paths
// of the operator (the tensor-core coupling in FP32, the double-float coupling
// generated once per block in FP64) run inside the solve.
//
// Outer loop (all precisions): r = b - A x with the FP64 operator; the columns
// whose true relative residual is at most rtol leave the block (the others are
// gathered into a compact block); an inner solve of A d = r for the remaining
// columns gives x += d.  With the FP64 operator the inner solve aims at the
// final tolerance; with the FP32 operator it stops at max(rtol |b|, delta |r|)
// (iterative refinement: the FP64 residual is recomputed after every inner
// solve, so the low-precision error does not accumulate).  Inner solvers:
// GMRES(restart) with two passes of classical Gram-Schmidt in FP64 and Givens
// rotations per column on the host (flexible GMRES, Saad 1993, for the learned
// preconditioner), or conjugate gradients.  All reductions are one CTA per
// (column, vector) with a fixed tree: deterministic.
#include <chrono>
#include <cmath>

#include "gmres_column.h"
#include "ibem_internal.cuh"

namespace ibem {

namespace {

inline unsigned nb_(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// out[k][r] = sum_i conj(V_k[r][i]) w[r][i] for k < nk (complex if CW = 2);
// V is [*][R][n CW], w is [R][n CW].  Grid (nk, R).
template <int CW>
__global__ void bdots_kernel(const double* __restrict__ V, int64_t n, int R, const double* __restrict__ w,
                             double* __restrict__ out) {
    __shared__ double sr[256], si[256];
    const int k = blockIdx.x, r = blockIdx.y;
    const double* v = V + ((int64_t)k * R + r) * n * CW;
    const double* x = w + (int64_t)r * n * CW;
    double ar = 0.0, ai = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        if (CW == 1) {
            ar += v[i] * x[i];
        } else {
            const double vr = v[2 * i], vi = v[2 * i + 1], xr = x[2 * i], xi = x[2 * i + 1];
            ar += vr * xr + vi * xi;
            ai += vr * xi - vi * xr;
        }
    }
    sr[threadIdx.x] = ar;
    si[threadIdx.x] = ai;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sr[threadIdx.x] += sr[threadIdx.x + s];
            si[threadIdx.x] += si[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * ((int64_t)k * R + r)] = sr[0];
        out[2 * ((int64_t)k * R + r) + 1] = si[0];
    }
}

// w[r] -= sum_{k < nk} V_k[r] h[k][r]   (h complex [nk][R][2]; real part only if CW = 1)
template <int CW>
__global__ void bgemv_sub_kernel(const double* __restrict__ V, int nk, int64_t n, int R,
                                 const double* __restrict__ h, double* __restrict__ w) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)R * n) return;
    const int r = (int)(idx / n);
    const int64_t i = idx % n;
    if (CW == 1) {
        double a = w[idx];
        for (int k = 0; k < nk; ++k) a -= V[((int64_t)k * R + r) * n + i] * h[2 * ((int64_t)k * R + r)];
        w[idx] = a;
    } else {
        double ar = w[2 * idx], ai = w[2 * idx + 1];
        for (int k = 0; k < nk; ++k) {
            const double* v = V + (((int64_t)k * R + r) * n + i) * 2;
            const double hr = h[2 * ((int64_t)k * R + r)], hi = h[2 * ((int64_t)k * R + r) + 1];
            ar -= v[0] * hr - v[1] * hi;
            ai -= v[0] * hi + v[1] * hr;
        }
        w[2 * idx] = ar;
        w[2 * idx + 1] = ai;
    }
}

// out[r] = sum_i a[r][i] b[r][i] over m doubles per column (real dot of the raw doubles)
__global__ void bdot_real_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t m,
                                 double* __restrict__ out) {
    __shared__ double s[256];
    const int r = blockIdx.x;
    const double* x = a + (int64_t)r * m;
    const double* y = b + (int64_t)r * m;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) acc += x[i] * y[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[r] = s[0];
}

// out[r][i] = s[r] * w[r][i]   (m doubles per column)
__global__ void bscale_kernel(const double* __restrict__ w, const double* __restrict__ s, int64_t m, int R,
                              double* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)R * m) return;
    out[idx] = s[idx / m] * w[idx];
}

// out[r] = sum_{k < nk} V_k[r] y[k][r]   (y complex [nk][R][2])
template <int CW>
__global__ void bcombine_kernel(const double* __restrict__ V, int nk, int64_t n, int R, const double* __restrict__ y,
                                double* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)R * n) return;
    const int r = (int)(idx / n);
    const int64_t i = idx % n;
    double ar = 0.0, ai = 0.0;
    for (int k = 0; k < nk; ++k) {
        const double yr = y[2 * ((int64_t)k * R + r)], yi = y[2 * ((int64_t)k * R + r) + 1];
        if (CW == 1) {
            ar += V[((int64_t)k * R + r) * n + i] * yr;
        } else {
            const double* v = V + (((int64_t)k * R + r) * n + i) * 2;
            ar += v[0] * yr - v[1] * yi;
            ai += v[0] * yi + v[1] * yr;
        }
    }
    if (CW == 1) {
        out[idx] = ar;
    } else {
        out[2 * idx] = ar;
        out[2 * idx + 1] = ai;
    }
}

// x[r] += a[r] p[r], rr[r] -= a[r] q[r] (CG update; m doubles per column)
__global__ void bcg_update_kernel(const double* __restrict__ a, const double* __restrict__ p,
                                  const double* __restrict__ q, int64_t m, int R, double* __restrict__ x,
                                  double* __restrict__ rr) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)R * m) return;
    const double al = a[idx / m];
    x[idx] += al * p[idx];
    rr[idx] -= al * q[idx];
}

// p[r] = z[r] + beta[r] p[r]
__global__ void bxpby_kernel(const double* __restrict__ z, const double* __restrict__ beta, int64_t m, int R,
                             double* __restrict__ p) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)R * m) return;
    p[idx] = z[idx] + beta[idx / m] * p[idx];
}

// y = a - b, y += x (m doubles)
__global__ void bsub_kernel(int64_t m, const double* __restrict__ a, const double* __restrict__ b,
                            double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) y[i] = a[i] - b[i];
}
__global__ void badd_kernel(int64_t m, const double* __restrict__ x, double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) y[i] += x[i];
}

// dst[j] = src[idx[j]] (column gather, m doubles per column); scatter: dst[idx[j]] = src[j]
__global__ void bgather_kernel(const double* __restrict__ src, const int* __restrict__ idx, int64_t m, int Ra,
                               double* __restrict__ dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)Ra * m) return;
    dst[t] = src[(int64_t)idx[t / m] * m + t % m];
}
__global__ void bscatter_kernel(const double* __restrict__ src, const int* __restrict__ idx, int64_t m, int Ra,
                                double* __restrict__ dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)Ra * m) return;
    dst[(int64_t)idx[t / m] * m + t % m] = src[t];
}

// point Jacobi for R columns: z[r][i] = v[r][i] / d[i] (complex division if CW = 2)
template <int CW>
__global__ void bjacobi_kernel(const double* __restrict__ v, const double* __restrict__ d, int64_t n, int R,
                               double* __restrict__ z) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)R * n) return;
    const int64_t i = idx % n;
    if (CW == 1) {
        z[idx] = d ? v[idx] / d[i] : v[idx];
    } else {
        const double vr = v[2 * idx], vi = v[2 * idx + 1];
        if (d) {
            const double dr = d[2 * i], di = d[2 * i + 1], den = dr * dr + di * di;
            z[2 * idx] = (vr * dr + vi * di) / den;
            z[2 * idx + 1] = (vi * dr - vr * di) / den;
        } else {
            z[2 * idx] = vr;
            z[2 * idx + 1] = vi;
        }
    }
}

struct Ctx {
    ibem_handle* h;
    int64_t n;      // dofs
    int CW;         // doubles per entry
    int64_t m;      // doubles per column = n CW
    cudaStream_t st;
    int precond;
    double* d_red = nullptr;    // device reduction scratch
    double* h_red = nullptr;    // pinned host copy
    size_t red_len = 0;
    std::vector<void*> owned;
    ~Ctx() {
        for (void* p : owned) cudaFreeAsync(p, st);
        if (h_red) cudaFreeHost(h_red);
    }
    template <typename T>
    cudaError_t alloc(T** p, size_t count) {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(p), count * sizeof(T) + 16, st);
        if (e == cudaSuccess) owned.push_back(*p);
        return e;
    }
    cudaError_t readback(size_t count, std::vector<double>& out) {
        cudaError_t e;
        if ((e = cudaMemcpyAsync(h_red, d_red, count * sizeof(double), cudaMemcpyDeviceToHost, st))) return e;
        if ((e = cudaStreamSynchronize(st))) return e;
        out.assign(h_red, h_red + count);
        return cudaSuccess;
    }
    cudaError_t upload(const std::vector<double>& v, double* dst) {
        std::copy(v.begin(), v.end(), h_red + red_len / 2);
        cudaError_t e = cudaMemcpyAsync(dst, h_red + red_len / 2, v.size() * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e) return e;
        return cudaStreamSynchronize(st);   // the pinned staging area is reused by the next upload
    }
    // squared 2-norms of R columns of x into out (host)
    cudaError_t norms2(const double* x, int R, std::vector<double>& out) {
        bdot_real_kernel<<<R, 256, 0, st>>>(x, x, m, d_red);
        return readback(R, out);
    }
    // z = M^-1 v for R columns (fixed preconditioners)
    cudaError_t precondition(const double* v, double* z, int R) {
        if (precond == IBEM_PRECOND_BLOCK_JACOBI || precond == IBEM_PRECOND_LEARNED) {
            for (int r = 0; r < R; ++r) {
                if (precond == IBEM_PRECOND_LEARNED) {
                    cudaError_t e = cnn_precondition(h, h->cnn, v + (size_t)r * m, z + (size_t)r * m);
                    if (e) return e;
                } else {
                    apply_block_jacobi(h, v + (size_t)r * m, z + (size_t)r * m);
                }
            }
            return cudaGetLastError();
        }
        const double* d = precond == IBEM_PRECOND_JACOBI ? h->d_diag : nullptr;
        if (CW == 1) bjacobi_kernel<1><<<nb_((int64_t)R * n, 256), 256, 0, st>>>(v, d, n, R, z);
        else bjacobi_kernel<2><<<nb_((int64_t)R * n, 256), 256, 0, st>>>(v, d, n, R, z);
        return cudaGetLastError();
    }
};

// One restart cycle of (flexible) GMRES on A_prec d = r for the Ra columns of r
// (x0 = 0), per-column absolute tolerances tol[]; adds the correction into d.
// its[] counts the Arnoldi steps of every column, *steps the operator
// applications.
ibem_status gmres_cycle(Ctx& c, int Ra, const double* r, double* d, const std::vector<double>& tol, int prec,
                        int restart, int max_steps, double* V, double* Z, double* w, double* tmp,
                        double* dh /* device [3][restart+1][Ra][2] */, std::vector<int>& its, int* steps) {
    ibem_handle* h = c.h;
    cudaStream_t st = c.st;
    const int m = restart;
    const int64_t M = c.m;
    const bool flex = c.precond == IBEM_PRECOND_LEARNED;
    std::vector<double> beta;
    if (c.norms2(r, Ra, beta) != cudaSuccess) return IBEM_ERR_CUDA;
    for (double& b : beta) b = std::sqrt(b);
    std::vector<char> active(Ra, 0);
    std::vector<int> kr(Ra, 0);
    std::vector<double> scale(Ra, 0.0);
    int nact = 0;
    for (int q = 0; q < Ra; ++q) {
        if (!std::isfinite(beta[q])) return IBEM_ERR_BREAKDOWN;
        active[q] = beta[q] > tol[q];
        nact += active[q];
        scale[q] = active[q] ? 1.0 / beta[q] : 0.0;
    }
    if (nact == 0) return IBEM_OK;
    if (c.upload(scale, c.d_red) != cudaSuccess) return IBEM_ERR_CUDA;
    bscale_kernel<<<nb_((int64_t)Ra * M, 256), 256, 0, st>>>(r, c.d_red, M, Ra, V);
    std::vector<GmresColumn> col(Ra);
    for (int q = 0; q < Ra; ++q) col[q].start(m, beta[q]);
    int j = 0;
    std::vector<double> hb, hq;
    for (; j < m && nact > 0 && *steps < max_steps; ++j) {
        double* Vj = V + (size_t)j * Ra * M;
        double* zj = flex ? Z + (size_t)j * Ra * M : tmp;
        if (c.precondition(Vj, zj, Ra) != cudaSuccess) return IBEM_ERR_CUDA;
        if (apply_operator(h, zj, w, Ra, prec) != cudaSuccess) return IBEM_ERR_CUDA;
        ++*steps;
        // two passes of classical Gram-Schmidt; coefficients of both passes and
        // the final norms come back in one read
        double* h0 = dh;
        double* h1 = dh + (size_t)2 * (j + 1) * Ra;
        double* hn = dh + (size_t)4 * (j + 1) * Ra;
        for (int pass = 0; pass < 2; ++pass) {
            double* hp = pass == 0 ? h0 : h1;
            if (c.CW == 1) {
                bdots_kernel<1><<<dim3(j + 1, Ra), 256, 0, st>>>(V, c.n, Ra, w, hp);
                bgemv_sub_kernel<1><<<nb_((int64_t)Ra * c.n, 256), 256, 0, st>>>(V, j + 1, c.n, Ra, hp, w);
            } else {
                bdots_kernel<2><<<dim3(j + 1, Ra), 256, 0, st>>>(V, c.n, Ra, w, hp);
                bgemv_sub_kernel<2><<<nb_((int64_t)Ra * c.n, 256), 256, 0, st>>>(V, j + 1, c.n, Ra, hp, w);
            }
        }
        bdot_real_kernel<<<Ra, 256, 0, st>>>(w, w, M, hn);
        if (cudaMemcpyAsync(c.h_red, dh, ((size_t)4 * (j + 1) * Ra + Ra) * sizeof(double), cudaMemcpyDeviceToHost, st) ||
            cudaStreamSynchronize(st))
            return IBEM_ERR_CUDA;
        hb.assign(c.h_red, c.h_red + (size_t)4 * (j + 1) * Ra + Ra);
        for (int q = 0; q < Ra; ++q) {
            scale[q] = 0.0;
            if (!active[q]) continue;
            hq.assign(2 * (j + 1), 0.0);
            for (int i = 0; i <= j; ++i) {
                hq[2 * i] = hb[2 * ((size_t)i * Ra + q)] + hb[(size_t)2 * (j + 1) * Ra + 2 * ((size_t)i * Ra + q)];
                hq[2 * i + 1] = hb[2 * ((size_t)i * Ra + q) + 1] +
                                hb[(size_t)2 * (j + 1) * Ra + 2 * ((size_t)i * Ra + q) + 1];
            }
            const double hnq = std::sqrt(hb[(size_t)4 * (j + 1) * Ra + q]);
            if (!std::isfinite(hnq)) return IBEM_ERR_BREAKDOWN;
            const double res = col[q].add(j, hq.data(), hnq);
            if (res < 0.0) return IBEM_ERR_BREAKDOWN;
            kr[q] = j + 1;
            ++its[q];
            if (res <= tol[q] || hnq == 0.0) {
                active[q] = 0;
                --nact;
            } else {
                scale[q] = 1.0 / hnq;
            }
        }
        // next basis vector (zero for finished columns)
        if (c.upload(scale, c.d_red) != cudaSuccess) return IBEM_ERR_CUDA;
        bscale_kernel<<<nb_((int64_t)Ra * M, 256), 256, 0, st>>>(w, c.d_red, M, Ra, V + (size_t)(j + 1) * Ra * M);
    }
    // back substitution per column, y [K][Ra][2] (zero beyond each column's k)
    const int K = j;
    if (K == 0) return IBEM_OK;
    std::vector<double> y((size_t)2 * K * Ra, 0.0), yy;
    for (int q = 0; q < Ra; ++q) {
        col[q].solve(yy);
        for (int i = 0; i < col[q].k; ++i) {
            y[2 * ((size_t)i * Ra + q)] = yy[2 * i];
            y[2 * ((size_t)i * Ra + q) + 1] = yy[2 * i + 1];
        }
    }
    if (c.upload(y, dh) != cudaSuccess) return IBEM_ERR_CUDA;
    const unsigned g1 = nb_((int64_t)Ra * c.n, 256);
    if (flex) {
        if (c.CW == 1) bcombine_kernel<1><<<g1, 256, 0, st>>>(Z, K, c.n, Ra, dh, tmp);
        else bcombine_kernel<2><<<g1, 256, 0, st>>>(Z, K, c.n, Ra, dh, tmp);
    } else {
        if (c.CW == 1) bcombine_kernel<1><<<g1, 256, 0, st>>>(V, K, c.n, Ra, dh, w);
        else bcombine_kernel<2><<<g1, 256, 0, st>>>(V, K, c.n, Ra, dh, w);
        if (c.precondition(w, tmp, Ra) != cudaSuccess) return IBEM_ERR_CUDA;
    }
    badd_kernel<<<nb_((int64_t)Ra * M, 256), 256, 0, st>>>((int64_t)Ra * M, tmp, d);
    return cudaGetLastError() ? IBEM_ERR_CUDA : IBEM_OK;
}

// Conjugate gradients on A_prec d = r for Ra real columns (d starts at 0),
// per-column absolute tolerances on the recursive residual.
ibem_status cg_block(Ctx& c, int Ra, const double* r, double* d, const std::vector<double>& tol, int prec,
                     int max_steps, double* rr, double* z, double* p, double* q, std::vector<int>& its, int* steps) {
    ibem_handle* h = c.h;
    cudaStream_t st = c.st;
    const int64_t M = c.m;
    const unsigned g1 = nb_((int64_t)Ra * M, 256);
    cudaMemsetAsync(d, 0, (size_t)Ra * M * sizeof(double), st);
    cudaMemcpyAsync(rr, r, (size_t)Ra * M * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (c.precondition(rr, z, Ra) != cudaSuccess) return IBEM_ERR_CUDA;
    cudaMemcpyAsync(p, z, (size_t)Ra * M * sizeof(double), cudaMemcpyDeviceToDevice, st);
    std::vector<double> rz, nrm, pq;
    bdot_real_kernel<<<Ra, 256, 0, st>>>(rr, z, M, c.d_red);
    if (c.readback(Ra, rz) != cudaSuccess) return IBEM_ERR_CUDA;
    if (c.norms2(rr, Ra, nrm) != cudaSuccess) return IBEM_ERR_CUDA;
    std::vector<char> active(Ra);
    int nact = 0;
    for (int k = 0; k < Ra; ++k) {
        active[k] = std::sqrt(nrm[k]) > tol[k];
        nact += active[k];
    }
    std::vector<double> al(Ra), be(Ra);
    while (nact > 0 && *steps < max_steps) {
        if (apply_operator(h, p, q, Ra, prec) != cudaSuccess) return IBEM_ERR_CUDA;
        ++*steps;
        bdot_real_kernel<<<Ra, 256, 0, st>>>(p, q, M, c.d_red);
        if (c.readback(Ra, pq) != cudaSuccess) return IBEM_ERR_CUDA;
        for (int k = 0; k < Ra; ++k) {
            al[k] = 0.0;
            if (!active[k]) continue;
            if (!(pq[k] > 0.0) || !std::isfinite(pq[k])) return IBEM_ERR_BREAKDOWN;
            al[k] = rz[k] / pq[k];
        }
        if (c.upload(al, c.d_red) != cudaSuccess) return IBEM_ERR_CUDA;
        bcg_update_kernel<<<g1, 256, 0, st>>>(c.d_red, p, q, M, Ra, d, rr);
        if (c.precondition(rr, z, Ra) != cudaSuccess) return IBEM_ERR_CUDA;
        bdot_real_kernel<<<Ra, 256, 0, st>>>(rr, rr, M, c.d_red);
        bdot_real_kernel<<<Ra, 256, 0, st>>>(rr, z, M, c.d_red + Ra);
        std::vector<double> both;
        if (c.readback(2 * Ra, both) != cudaSuccess) return IBEM_ERR_CUDA;
        for (int k = 0; k < Ra; ++k) {
            be[k] = 0.0;
            if (!active[k]) continue;
            ++its[k];
            if (!std::isfinite(both[k])) return IBEM_ERR_BREAKDOWN;
            if (std::sqrt(both[k]) <= tol[k]) {
                active[k] = 0;
                --nact;
                continue;
            }
            be[k] = both[Ra + k] / rz[k];
            rz[k] = both[Ra + k];
        }
        if (c.upload(be, c.d_red) != cudaSuccess) return IBEM_ERR_CUDA;
        bxpby_kernel<<<g1, 256, 0, st>>>(z, c.d_red, M, Ra, p);
    }
    return cudaGetLastError() ? IBEM_ERR_CUDA : IBEM_OK;
}

}  // namespace

ibem_status solve_block_impl(ibem_handle* h, const double* b, double* x, int R, double rtol, int maxit,
                             int precond, int precision, ibem_solve_info* info) {
    auto t0 = std::chrono::steady_clock::now();
    Ctx c;
    c.h = h;
    c.n = h->P.N;
    c.CW = h->helm ? 2 : 1;
    c.m = c.n * c.CW;
    c.st = h->stream;
    c.precond = precond;
    cudaStream_t st = h->stream;
    const int restart = 100;
    const int64_t M = c.m;
    // reduction scratch: dots of a full cycle (3 (restart + 1) R complex)
    const size_t red = (size_t)6 * (restart + 2) * R + 64;
    c.red_len = 2 * red;
    if (cudaMallocHost(&c.h_red, c.red_len * sizeof(double)) != cudaSuccess) return IBEM_ERR_OOM;
    if (c.alloc(&c.d_red, red)) return IBEM_ERR_OOM;
    double *dh = nullptr, *rb = nullptr, *xb = nullptr, *bb = nullptr, *dd = nullptr, *w = nullptr, *tmp = nullptr;
    double *V = nullptr, *Z = nullptr;
    int* d_idx = nullptr;
    const size_t blk = (size_t)R * M;
    if (c.alloc(&dh, (size_t)6 * (restart + 2) * R) || c.alloc(&rb, blk) || c.alloc(&xb, blk) || c.alloc(&bb, blk) ||
        c.alloc(&dd, blk) || c.alloc(&w, blk) || c.alloc(&tmp, blk) || c.alloc(&d_idx, (size_t)R))
        return IBEM_ERR_OOM;
    const bool gm = h->helm;
    if (gm) {
        if (c.alloc(&V, (size_t)(restart + 1) * blk)) return IBEM_ERR_OOM;
        if (precond == IBEM_PRECOND_LEARNED && c.alloc(&Z, (size_t)restart * blk)) return IBEM_ERR_OOM;
    } else if (c.alloc(&V, 3 * blk)) {   // CG: z, p, q
        return IBEM_ERR_OOM;
    }
    // norms of b; columns with b = 0 get x = 0
    std::vector<double> nb;
    if (c.norms2(b, R, nb) != cudaSuccess) return IBEM_ERR_CUDA;
    cudaMemsetAsync(x, 0, blk * sizeof(double), st);
    std::vector<int> act;
    std::vector<double> tol_final(R);
    for (int r = 0; r < R; ++r) {
        nb[r] = std::sqrt(nb[r]);
        if (!std::isfinite(nb[r])) return IBEM_ERR_BREAKDOWN;   // NaN or Inf in the right-hand side
        tol_final[r] = rtol * nb[r];
        if (nb[r] > 0.0) act.push_back(r);
    }
    std::vector<int> its(R, 0);
    int steps = 0, outer = 0;
    ibem_status status = IBEM_OK;
    const double delta = precision == IBEM_FP32 ? 1e-3 : 0.0;
    const int prec = precision == IBEM_FP32 ? IBEM_FP32 : IBEM_FP64;
    std::vector<double> rn;
    // compact block of the active columns: b, x (zero) and the residual r = b
    auto gather = [&](const std::vector<int>& a) -> bool {
        std::vector<int> tmpi(a.begin(), a.end());
        if (cudaMemcpyAsync(d_idx, tmpi.data(), tmpi.size() * sizeof(int), cudaMemcpyHostToDevice, st) ||
            cudaStreamSynchronize(st))
            return false;
        const unsigned ga = nb_((int64_t)a.size() * M, 256);
        bgather_kernel<<<ga, 256, 0, st>>>(b, d_idx, M, (int)a.size(), bb);
        bgather_kernel<<<ga, 256, 0, st>>>(x, d_idx, M, (int)a.size(), xb);
        return cudaGetLastError() == cudaSuccess;
    };
    if (!act.empty()) {
        if (!gather(act)) return IBEM_ERR_CUDA;
        cudaMemcpyAsync(rb, bb, act.size() * M * sizeof(double), cudaMemcpyDeviceToDevice, st);
    }
    while (!act.empty()) {
        int Ra = (int)act.size();
        if (c.norms2(rb, Ra, rn) != cudaSuccess) return IBEM_ERR_CUDA;
        std::vector<int> keep;
        std::vector<double> tol;
        for (int k = 0; k < Ra; ++k) {
            const double v = std::sqrt(rn[k]);
            if (!std::isfinite(v)) return IBEM_ERR_BREAKDOWN;
            if (v > tol_final[act[k]]) {
                keep.push_back(k);
                tol.push_back(std::max(tol_final[act[k]], delta * v));
            }
        }
        if (keep.empty()) break;
        if (steps >= maxit) {
            status = IBEM_ERR_NOCONV;
            break;
        }
        if ((int)keep.size() < Ra) {
            // drop the converged columns: residuals from the old compact block,
            // b and x from the full arrays
            std::vector<int> kk(keep.begin(), keep.end());
            if (cudaMemcpyAsync(d_idx, kk.data(), kk.size() * sizeof(int), cudaMemcpyHostToDevice, st) ||
                cudaStreamSynchronize(st))
                return IBEM_ERR_CUDA;
            bgather_kernel<<<nb_((int64_t)kk.size() * M, 256), 256, 0, st>>>(rb, d_idx, M, (int)kk.size(), tmp);
            cudaMemcpyAsync(rb, tmp, kk.size() * M * sizeof(double), cudaMemcpyDeviceToDevice, st);
            std::vector<int> nact;
            for (int k : keep) nact.push_back(act[k]);
            act = nact;
            Ra = (int)act.size();
            if (!gather(act)) return IBEM_ERR_CUDA;
        } else if (cudaMemcpyAsync(d_idx, act.data(), act.size() * sizeof(int), cudaMemcpyHostToDevice, st) ||
                   cudaStreamSynchronize(st)) {
            return IBEM_ERR_CUDA;
        }
        ++outer;
        std::vector<int> its_a(Ra, 0);
        cudaMemsetAsync(dd, 0, (size_t)Ra * M * sizeof(double), st);
        ibem_status s;
        if (gm) s = gmres_cycle(c, Ra, rb, dd, tol, prec, restart, maxit, V, Z, w, tmp, dh, its_a, &steps);
        else s = cg_block(c, Ra, rb, dd, tol, prec, maxit, V, V + blk, V + 2 * blk, w, its_a, &steps);
        if (s != IBEM_OK) {
            status = s;
            break;
        }
        for (int k = 0; k < Ra; ++k) its[act[k]] += its_a[k];
        // x += d; r = b - A x with the FP64 operator
        const unsigned ga = nb_((int64_t)Ra * M, 256);
        badd_kernel<<<ga, 256, 0, st>>>((int64_t)Ra * M, dd, xb);
        bscatter_kernel<<<ga, 256, 0, st>>>(xb, d_idx, M, Ra, x);
        if (apply_operator(h, xb, w, Ra, IBEM_FP64) != cudaSuccess) return IBEM_ERR_CUDA;
        bsub_kernel<<<ga, 256, 0, st>>>((int64_t)Ra * M, bb, w, rb);
    }
    // true residuals of all columns with the FP64 operator
    double worst = 0.0;
    int total = 0;
    if (status == IBEM_OK || status == IBEM_ERR_NOCONV) {
        if (apply_operator(h, x, tmp, R, IBEM_FP64) != cudaSuccess) return IBEM_ERR_CUDA;
        bsub_kernel<<<nb_((int64_t)R * M, 256), 256, 0, st>>>((int64_t)R * M, b, tmp, w);
        if (c.norms2(w, R, rn) != cudaSuccess) return IBEM_ERR_CUDA;
        for (int r = 0; r < R; ++r)
            if (nb[r] > 0.0) worst = std::max(worst, std::sqrt(rn[r]) / nb[r]);
        if (status == IBEM_OK && worst > rtol * 1.0001) status = IBEM_ERR_NOCONV;
    }
    for (int v : its) total += v;
    if (info) {
        info->iterations = total;
        info->outer = outer;
        info->rel_residual = worst;
        info->steps = steps;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    cudaStreamSynchronize(st);
    return status;
}

}  // namespace ibem
