// Krylov solvers of libibem (Sec. 4 item 3): Jacobi-preconditioned conjugate
// gradients on T A T^T w = b for the Laplace single layer (symmetric positive
// definite), either on the FP64 operator or on the FP32 operator with reliable
// updates of the residual by the FP64 operator.
//
// Vectors are FP64.  Reductions run in one CTA per call (N is at most a few
// 10^5 here), so every dot product is deterministic.
#include <chrono>
#include <cmath>

#include "ibem_internal.cuh"

namespace ibem {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// out[0] = sum a[i] * b[i]
__global__ void dot_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                           double* __restrict__ out) {
    __shared__ double s[1024];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += a[i] * b[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = s[0];
}

// x += alpha p; r -= alpha Ap; z = r / d; out = (r.r, r.z)
__global__ void cg_update_kernel(int64_t n, const double* __restrict__ alpha_p, double* __restrict__ x,
                                 double* __restrict__ r, const double* __restrict__ p,
                                 const double* __restrict__ Ap, const double* __restrict__ d,
                                 double* __restrict__ z, double* __restrict__ out) {
    __shared__ double s1[1024], s2[1024];
    double alpha = alpha_p[0];
    double a1 = 0.0, a2 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        x[i] += alpha * p[i];
        double ri = r[i] - alpha * Ap[i];
        r[i] = ri;
        double zi = d ? ri / d[i] : ri;
        z[i] = zi;
        a1 += ri * ri;
        a2 += ri * zi;
    }
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = s1[0]; out[1] = s2[0]; }
}

__global__ void scal_div_kernel(int64_t n, const double* __restrict__ r, const double* __restrict__ d,
                                double* __restrict__ z) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = d ? r[i] / d[i] : r[i];
}

// p = z + beta p
__global__ void xpby_kernel(int64_t n, const double* __restrict__ z, double beta, double* __restrict__ p) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = z[i] + beta * p[i];
}

// y = a - b
__global__ void sub_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a[i] - b[i];
}

// y += x
__global__ void add_kernel(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += x[i];
}

// ---- complex vectors (interleaved re, im) for GMRES ---------------------------------
// out[2k], out[2k+1] = sum_i conj(V[k][i]) w[i] for k = 0..nk-1 (one CTA per k)
__global__ void zdots_kernel(const double* __restrict__ V, int64_t N, const double* __restrict__ w, int nk,
                             double* __restrict__ out) {
    __shared__ double sr[256], si[256];
    const double* v = V + (int64_t)blockIdx.x * 2 * N;
    double ar = 0.0, ai = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        double vr = v[2 * i], vi = v[2 * i + 1], xr = w[2 * i], xi = w[2 * i + 1];
        ar += vr * xr + vi * xi;
        ai += vr * xi - vi * xr;
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
        out[2 * blockIdx.x] = sr[0];
        out[2 * blockIdx.x + 1] = si[0];
    }
}

// w -= sum_k V[k] h[k]   (complex)
__global__ void zgemv_sub_kernel(const double* __restrict__ V, int64_t N, const double* __restrict__ h, int nk,
                                 double* __restrict__ w) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double ar = w[2 * i], ai = w[2 * i + 1];
    for (int k = 0; k < nk; ++k) {
        double vr = V[(int64_t)k * 2 * N + 2 * i], vi = V[(int64_t)k * 2 * N + 2 * i + 1];
        double hr = h[2 * k], hi = h[2 * k + 1];
        ar -= vr * hr - vi * hi;
        ai -= vr * hi + vi * hr;
    }
    w[2 * i] = ar;
    w[2 * i + 1] = ai;
}

// out = (sum_k V[k] y[k]) / d   (complex; d = Jacobi diagonal or null)
__global__ void zcombine_kernel(const double* __restrict__ V, int64_t N, const double* __restrict__ y, int nk,
                                const double* __restrict__ d, double* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double ar = 0.0, ai = 0.0;
    for (int k = 0; k < nk; ++k) {
        double vr = V[(int64_t)k * 2 * N + 2 * i], vi = V[(int64_t)k * 2 * N + 2 * i + 1];
        ar += vr * y[2 * k] - vi * y[2 * k + 1];
        ai += vr * y[2 * k + 1] + vi * y[2 * k];
    }
    if (d) {
        double dr = d[2 * i], di = d[2 * i + 1], den = dr * dr + di * di;
        double br = (ar * dr + ai * di) / den, bi = (ai * dr - ar * di) / den;
        ar = br;
        ai = bi;
    }
    out[2 * i] = ar;
    out[2 * i + 1] = ai;
}

// z = v / d (complex), or copy
__global__ void zdiv_kernel(int64_t N, const double* __restrict__ v, const double* __restrict__ d,
                            double* __restrict__ z) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double vr = v[2 * i], vi = v[2 * i + 1];
    if (d) {
        double dr = d[2 * i], di = d[2 * i + 1], den = dr * dr + di * di;
        z[2 * i] = (vr * dr + vi * di) / den;
        z[2 * i + 1] = (vi * dr - vr * di) / den;
    } else {
        z[2 * i] = vr;
        z[2 * i + 1] = vi;
    }
}

// y = alpha * x (real alpha), n doubles
__global__ void dscal_copy_kernel(int64_t n, double alpha, const double* __restrict__ x, double* __restrict__ y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = alpha * x[i];
}

namespace {

struct Work {
    double *r, *z, *p, *Ap, *x, *d, *rr;
};

cudaError_t readback(ibem_handle* h, const double* dev, int n, double* host) {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(h->h_red, dev, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream))) return e;
    if ((e = cudaStreamSynchronize(h->stream))) return e;
    for (int i = 0; i < n; ++i) host[i] = h->h_red[i];
    return cudaSuccess;
}

cudaError_t norm2(ibem_handle* h, const double* v, int64_t n, double* out) {
    dot_kernel<<<1, 1024, 0, h->stream>>>(v, v, n, h->d_red);
    double s;
    cudaError_t e = readback(h, h->d_red, 1, &s);
    *out = std::sqrt(s);
    return e;
}

// CG on A (precision prec) for A x = b, x starts at 0.  Stops when
// |r_k| <= tol_abs (recurrence residual).  Returns iterations in *its.
ibem_status cg(ibem_handle* h, const double* b, double* x, const Work& w, int prec, double tol_abs,
               int maxit, int precond, int* its) {
    Plan& P = h->P;
    int64_t N = P.N;
    cudaStream_t st = h->stream;
    const double* d = precond == IBEM_PRECOND_JACOBI ? h->d_diag : nullptr;
    const bool block = precond == IBEM_PRECOND_BLOCK_JACOBI;
    cudaMemsetAsync(x, 0, N * sizeof(double), st);
    cudaMemcpyAsync(w.r, b, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    scal_div_kernel<<<nblk(N, 256), 256, 0, st>>>(N, w.r, d, w.z);
    if (block) apply_block_jacobi(h, w.r, w.z);
    cudaMemcpyAsync(w.p, w.z, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    dot_kernel<<<1, 1024, 0, st>>>(w.r, w.z, N, h->d_red);
    double rz;
    if (readback(h, h->d_red, 1, &rz) != cudaSuccess) return IBEM_ERR_CUDA;
    *its = 0;
    if (std::sqrt(std::fabs(rz)) == 0.0) return IBEM_OK;
    for (int it = 1; it <= maxit; ++it) {
        if (apply_operator(h, w.p, w.Ap, 1, prec) != cudaSuccess) return IBEM_ERR_CUDA;
        dot_kernel<<<1, 1024, 0, st>>>(w.p, w.Ap, N, h->d_red);
        double pAp;
        if (readback(h, h->d_red, 1, &pAp) != cudaSuccess) return IBEM_ERR_CUDA;
        if (!(pAp > 0.0) || !std::isfinite(pAp)) { *its = it; return IBEM_ERR_BREAKDOWN; }
        h->h_red[0] = rz / pAp;
        cudaMemcpyAsync(h->d_red + 2, h->h_red, sizeof(double), cudaMemcpyHostToDevice, st);
        cg_update_kernel<<<1, 1024, 0, st>>>(N, h->d_red + 2, x, w.r, w.p, w.Ap, d, w.z, h->d_red);
        double rr[2];
        if (readback(h, h->d_red, 2, rr) != cudaSuccess) return IBEM_ERR_CUDA;
        *its = it;
        if (!std::isfinite(rr[0])) return IBEM_ERR_BREAKDOWN;
        if (std::sqrt(rr[0]) <= tol_abs) return IBEM_OK;
        if (block) {
            apply_block_jacobi(h, w.r, w.z);
            dot_kernel<<<1, 1024, 0, st>>>(w.r, w.z, N, h->d_red);
            if (readback(h, h->d_red, 1, &rr[1]) != cudaSuccess) return IBEM_ERR_CUDA;
        }
        double beta = rr[1] / rz;
        rz = rr[1];
        xpby_kernel<<<nblk(N, 256), 256, 0, st>>>(N, w.z, beta, w.p);
    }
    return IBEM_ERR_NOCONV;
}

// Mixed precision: conjugate gradients whose operator is the FP32 operator,
// with reliable updates (Sleijpen and van der Vorst): whenever the recursively
// updated residual has dropped by `drop` since the last update, or looks
// converged, it is replaced by the true residual b - A64 x computed with the
// FP64 operator, and the search direction is kept.  Convergence is decided on
// the true residual only.  *updates counts the FP64 applications.
ibem_status cg_reliable(ibem_handle* h, const double* b, double* x, const Work& w, double tol_abs, int maxit,
                        int precond, int* its, int* updates) {
    Plan& P = h->P;
    int64_t N = P.N;
    cudaStream_t st = h->stream;
    const double* d = precond == IBEM_PRECOND_JACOBI ? h->d_diag : nullptr;
    const bool block = precond == IBEM_PRECOND_BLOCK_JACOBI;
    const double drop = 1e-2;
    cudaMemsetAsync(x, 0, N * sizeof(double), st);
    cudaMemcpyAsync(w.r, b, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    scal_div_kernel<<<nblk(N, 256), 256, 0, st>>>(N, w.r, d, w.z);
    if (block) apply_block_jacobi(h, w.r, w.z);
    cudaMemcpyAsync(w.p, w.z, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    dot_kernel<<<1, 1024, 0, st>>>(w.r, w.z, N, h->d_red);
    double rz;
    if (readback(h, h->d_red, 1, &rz) != cudaSuccess) return IBEM_ERR_CUDA;
    double ref;
    if (norm2(h, w.r, N, &ref) != cudaSuccess) return IBEM_ERR_CUDA;
    *its = 0;
    *updates = 0;
    if (ref <= tol_abs) return IBEM_OK;
    for (int it = 1; it <= maxit; ++it) {
        if (apply_operator(h, w.p, w.Ap, 1, IBEM_FP32) != cudaSuccess) return IBEM_ERR_CUDA;
        dot_kernel<<<1, 1024, 0, st>>>(w.p, w.Ap, N, h->d_red);
        double pAp;
        if (readback(h, h->d_red, 1, &pAp) != cudaSuccess) return IBEM_ERR_CUDA;
        if (!(pAp > 0.0) || !std::isfinite(pAp)) { *its = it; return IBEM_ERR_BREAKDOWN; }
        h->h_red[0] = rz / pAp;
        cudaMemcpyAsync(h->d_red + 2, h->h_red, sizeof(double), cudaMemcpyHostToDevice, st);
        cg_update_kernel<<<1, 1024, 0, st>>>(N, h->d_red + 2, x, w.r, w.p, w.Ap, d, w.z, h->d_red);
        double rr[2];
        if (readback(h, h->d_red, 2, rr) != cudaSuccess) return IBEM_ERR_CUDA;
        *its = it;
        if (!std::isfinite(rr[0])) return IBEM_ERR_BREAKDOWN;
        double rn = std::sqrt(rr[0]);
        double rz_new = rr[1];
        if (rn <= drop * ref || rn <= tol_abs) {
            if (apply_operator(h, x, w.Ap, 1, IBEM_FP64) != cudaSuccess) return IBEM_ERR_CUDA;
            ++*updates;
            sub_kernel<<<nblk(N, 256), 256, 0, st>>>(N, b, w.Ap, w.r);
            if (norm2(h, w.r, N, &rn) != cudaSuccess) return IBEM_ERR_CUDA;
            ref = rn;
            if (rn <= tol_abs) return IBEM_OK;
            scal_div_kernel<<<nblk(N, 256), 256, 0, st>>>(N, w.r, d, w.z);
            if (block) apply_block_jacobi(h, w.r, w.z);
            dot_kernel<<<1, 1024, 0, st>>>(w.r, w.z, N, h->d_red);
            if (readback(h, h->d_red, 1, &rz_new) != cudaSuccess) return IBEM_ERR_CUDA;
        } else if (block) {
            apply_block_jacobi(h, w.r, w.z);
            dot_kernel<<<1, 1024, 0, st>>>(w.r, w.z, N, h->d_red);
            if (readback(h, h->d_red, 1, &rz_new) != cudaSuccess) return IBEM_ERR_CUDA;
        }
        double beta = rz_new / rz;
        rz = rz_new;
        xpby_kernel<<<nblk(N, 256), 256, 0, st>>>(N, w.z, beta, w.p);
    }
    return IBEM_ERR_NOCONV;
}

// Restarted GMRES with right Jacobi preconditioning for the complex-symmetric
// Helmholtz matrix.  Arnoldi with two passes of classical Gram-Schmidt in FP64;
// Givens rotations on the host.  The Arnoldi operator has precision `prec`;
// every restart recomputes the residual b - A x with the FP64 operator, so with
// prec = IBEM_FP32 the restarts are FP64 residual corrections.
// Iterates of the first GMRES cycle kept for residual/error training pairs:
// after step j with (j + 1) % stride == 0 the iterate x_j goes to X[n] and its
// residual r_j = b - A x_j to R[n], the latter from the Arnoldi relation
// r_j = V_{j+1} (beta e_1 - Hbar_j y_j) without an operator application.
struct Recorder {
    int stride = 1, max = 0, n = 0;
    double* X = nullptr;  // [max][2N], or null: iterates not kept
    double* R = nullptr;  // [max][2N]
};

ibem_status gmres(ibem_handle* h, const double* b, double* x, double tol_abs, int maxit, int precond, int prec,
                  int restart, int* its, int* restarts, Recorder* rec = nullptr) {
    Plan& P = h->P;
    const int64_t N = P.N;
    cudaStream_t st = h->stream;
    const double* d = precond == IBEM_PRECOND_JACOBI ? h->d_diag : nullptr;
    const bool block = precond == IBEM_PRECOND_BLOCK_JACOBI;
    // flexible GMRES (Saad 1993) for the learned preconditioner, which is not a
    // fixed linear map: the preconditioned vectors Z are kept and x += Z y
    const bool flex = precond == IBEM_PRECOND_LEARNED;
    const int m = restart;
    double *V = nullptr, *w = nullptr, *z = nullptr, *hv = nullptr, *Z = nullptr;
    if (flex && cudaMallocAsync(&Z, (size_t)m * 2 * N * sizeof(double), st) != cudaSuccess) return IBEM_ERR_OOM;
    if (cudaMallocAsync(&V, (size_t)(m + 1) * 2 * N * sizeof(double), st) != cudaSuccess) return IBEM_ERR_OOM;
    if (cudaMallocAsync(&w, (size_t)2 * N * sizeof(double), st) != cudaSuccess) return IBEM_ERR_OOM;
    if (cudaMallocAsync(&z, (size_t)2 * N * sizeof(double), st) != cudaSuccess) return IBEM_ERR_OOM;
    if (cudaMallocAsync(&hv, (size_t)2 * (m + 1) * sizeof(double), st) != cudaSuccess) return IBEM_ERR_OOM;
    std::vector<double> H((size_t)(m + 1) * m * 2, 0.0), cs(m), snr(m), sni(m), g(2 * (m + 1)), hh(2 * (m + 1));
    std::vector<double> Hu(rec ? (size_t)(m + 1) * m * 2 : 0, 0.0);   // unrotated Hessenberg (recording)
    ibem_status status = IBEM_ERR_NOCONV;
    *its = 0;
    *restarts = 0;
    auto done = [&](ibem_status s) {
        cudaFreeAsync(V, st);
        cudaFreeAsync(w, st);
        cudaFreeAsync(z, st);
        cudaFreeAsync(hv, st);
        if (Z) cudaFreeAsync(Z, st);
        cudaStreamSynchronize(st);
        return s;
    };
    cudaMemsetAsync(x, 0, 2 * N * sizeof(double), st);
    cudaMemcpyAsync(w, b, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    auto Hr = [&](int i, int j) -> double& { return H[2 * ((size_t)i * m + j)]; };
    auto Hi = [&](int i, int j) -> double& { return H[2 * ((size_t)i * m + j) + 1]; };
    const unsigned nb = nblk(N, 256);
    // back substitution R y = g (complex, upper triangular k x k)
    auto backsolve = [&](int k, std::vector<double>& y) {
        y.assign(2 * k, 0.0);
        for (int i = k - 1; i >= 0; --i) {
            double sr = g[2 * i], si = g[2 * i + 1];
            for (int l = i + 1; l < k; ++l) {
                sr -= Hr(i, l) * y[2 * l] - Hi(i, l) * y[2 * l + 1];
                si -= Hr(i, l) * y[2 * l + 1] + Hi(i, l) * y[2 * l];
            }
            double dr = Hr(i, i), di = Hi(i, i), den = dr * dr + di * di;
            y[2 * i] = (sr * dr + si * di) / den;
            y[2 * i + 1] = (si * dr - sr * di) / den;
        }
    };
    // M^-1 (V y) into out (tmp is scratch), for the fixed preconditioners
    auto precond_combine = [&](int k, double* tmp, double* out) {
        if (flex) {
            zcombine_kernel<<<nb, 256, 0, st>>>(Z, N, hv, k, nullptr, out);
        } else if (block) {
            zcombine_kernel<<<nb, 256, 0, st>>>(V, N, hv, k, nullptr, tmp);
            apply_block_jacobi(h, tmp, out);
        } else {
            zcombine_kernel<<<nb, 256, 0, st>>>(V, N, hv, k, d, out);
        }
    };
    while (*its < maxit) {
        double beta;
        if (norm2(h, w, 2 * N, &beta) != cudaSuccess) return done(IBEM_ERR_CUDA);
        if (!std::isfinite(beta)) return done(IBEM_ERR_BREAKDOWN);
        if (beta <= tol_abs) { status = IBEM_OK; break; }
        dscal_copy_kernel<<<nblk(2 * N, 256), 256, 0, st>>>(2 * N, 1.0 / beta, w, V);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m && *its < maxit; ++j) {
            double* zj = flex ? Z + (size_t)j * 2 * N : z;
            if (flex) {
                if (cnn_precondition(h, h->cnn, V + (size_t)j * 2 * N, zj) != cudaSuccess) return done(IBEM_ERR_CUDA);
            } else if (block) {
                apply_block_jacobi(h, V + (size_t)j * 2 * N, zj);
            } else {
                zdiv_kernel<<<nb, 256, 0, st>>>(N, V + (size_t)j * 2 * N, d, zj);
            }
            if (apply_operator(h, zj, w, 1, prec) != cudaSuccess) return done(IBEM_ERR_CUDA);
            for (int i = 0; i <= j; ++i) { Hr(i, j) = 0.0; Hi(i, j) = 0.0; }
            for (int pass = 0; pass < 2; ++pass) {
                zdots_kernel<<<j + 1, 256, 0, st>>>(V, N, w, j + 1, hv);
                zgemv_sub_kernel<<<nb, 256, 0, st>>>(V, N, hv, j + 1, w);
                if (cudaMemcpyAsync(hh.data(), hv, 2 * (j + 1) * sizeof(double), cudaMemcpyDeviceToHost, st) ||
                    cudaStreamSynchronize(st))
                    return done(IBEM_ERR_CUDA);
                for (int i = 0; i <= j; ++i) { Hr(i, j) += hh[2 * i]; Hi(i, j) += hh[2 * i + 1]; }
            }
            double hn;
            if (norm2(h, w, 2 * N, &hn) != cudaSuccess) return done(IBEM_ERR_CUDA);
            Hr(j + 1, j) = hn;
            Hi(j + 1, j) = 0.0;
            if (rec)
                for (int i = 0; i <= j + 1; ++i) {
                    Hu[2 * ((size_t)i * m + j)] = Hr(i, j);
                    Hu[2 * ((size_t)i * m + j) + 1] = Hi(i, j);
                }
            if (hn != 0.0)
                dscal_copy_kernel<<<nblk(2 * N, 256), 256, 0, st>>>(2 * N, 1.0 / hn, w, V + (size_t)(j + 1) * 2 * N);
            // apply the previous rotations to column j
            for (int i = 0; i < j; ++i) {
                double ar = Hr(i, j), ai = Hi(i, j), br = Hr(i + 1, j), bi = Hi(i + 1, j);
                // [c  s; -conj(s)  c] with real c, complex s
                Hr(i, j) = cs[i] * ar + (snr[i] * br - sni[i] * bi);
                Hi(i, j) = cs[i] * ai + (snr[i] * bi + sni[i] * br);
                Hr(i + 1, j) = -(snr[i] * ar + sni[i] * ai) + cs[i] * br;
                Hi(i + 1, j) = -(snr[i] * ai - sni[i] * ar) + cs[i] * bi;
            }
            // new rotation zeroing H(j+1, j)
            double ar = Hr(j, j), ai = Hi(j, j), bb = Hr(j + 1, j);
            double na = std::sqrt(ar * ar + ai * ai);
            double den = std::sqrt(na * na + bb * bb);
            if (den == 0.0) return done(IBEM_ERR_BREAKDOWN);
            if (na == 0.0) { cs[j] = 0.0; snr[j] = 1.0; sni[j] = 0.0; }
            else {
                cs[j] = na / den;
                // s = (a / |a|) * conj(b) / den, b real
                snr[j] = (ar / na) * bb / den;
                sni[j] = (ai / na) * bb / den;
            }
            Hr(j, j) = cs[j] * ar + (snr[j] * bb);
            Hi(j, j) = cs[j] * ai + (sni[j] * bb);
            Hr(j + 1, j) = 0.0;
            Hi(j + 1, j) = 0.0;
            double gr = g[2 * j], gi = g[2 * j + 1];
            g[2 * j] = cs[j] * gr;
            g[2 * j + 1] = cs[j] * gi;
            g[2 * (j + 1)] = -(snr[j] * gr + sni[j] * gi);
            g[2 * (j + 1) + 1] = -(snr[j] * gi - sni[j] * gr);
            k = j + 1;
            ++*its;
            double res = std::sqrt(g[2 * k] * g[2 * k] + g[2 * k + 1] * g[2 * k + 1]);
            if (!std::isfinite(res)) return done(IBEM_ERR_BREAKDOWN);
            if (rec && *restarts == 0 && rec->n < rec->max && k % rec->stride == 0) {
                // x_k = M^-1 V_k y_k (x0 = 0 in the first cycle)
                std::vector<double> y, c(2 * (k + 1), 0.0);
                backsolve(k, y);
                if (cudaMemcpyAsync(hv, y.data(), 2 * k * sizeof(double), cudaMemcpyHostToDevice, st))
                    return done(IBEM_ERR_CUDA);
                if (rec->X) precond_combine(k, w, rec->X + (size_t)rec->n * 2 * N);
                // r_k = V_{k+1} (beta e_1 - Hbar_k y_k)
                c[0] = beta;
                for (int i = 0; i <= k; ++i)
                    for (int l = 0; l < k; ++l) {
                        if (i > l + 1) continue;
                        const double hr = Hu[2 * ((size_t)i * m + l)], hi = Hu[2 * ((size_t)i * m + l) + 1];
                        c[2 * i] -= hr * y[2 * l] - hi * y[2 * l + 1];
                        c[2 * i + 1] -= hr * y[2 * l + 1] + hi * y[2 * l];
                    }
                if (cudaMemcpyAsync(hv, c.data(), 2 * (k + 1) * sizeof(double), cudaMemcpyHostToDevice, st))
                    return done(IBEM_ERR_CUDA);
                zcombine_kernel<<<nb, 256, 0, st>>>(V, N, hv, hn != 0.0 ? k + 1 : k, nullptr,
                                                    rec->R + (size_t)rec->n * 2 * N);
                ++rec->n;
            }
            if (res <= tol_abs || hn == 0.0) break;
        }
        std::vector<double> y;
        backsolve(k, y);
        if (cudaMemcpyAsync(hv, y.data(), 2 * k * sizeof(double), cudaMemcpyHostToDevice, st))
            return done(IBEM_ERR_CUDA);
        precond_combine(k, w, z);
        add_kernel<<<nblk(2 * N, 256), 256, 0, st>>>(2 * N, z, x);
        // restart residual with the FP64 operator
        if (apply_operator(h, x, w, 1, IBEM_FP64) != cudaSuccess) return done(IBEM_ERR_CUDA);
        sub_kernel<<<nblk(2 * N, 256), 256, 0, st>>>(2 * N, b, w, w);
        ++*restarts;
    }
    if (status != IBEM_OK) {
        double beta;
        if (norm2(h, w, 2 * N, &beta) == cudaSuccess && beta <= tol_abs) status = IBEM_OK;
    }
    return done(status);
}

// Training images of one pair: in = s / sigma, target = (x* - x - s) / sigma,
// sigma^2 = |s|^2 / (2N) (ss[0] = |s|^2), patch images [npatch][2][n1][n1].
__global__ void pair_images_kernel(int64_t N, int n1, const double* __restrict__ xstar, const double* __restrict__ x,
                                   const double* __restrict__ s, const double* __restrict__ ss,
                                   float* __restrict__ in_img, float* __restrict__ tgt_img) {
    int64_t dof = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (dof >= N) return;
    const int64_t per = (int64_t)n1 * n1;
    const int64_t patch = dof / per, pix = dof % per;
    const double inv = ss[0] > 0.0 ? 1.0 / sqrt(ss[0] / (2.0 * N)) : 0.0;
    for (int c = 0; c < 2; ++c) {
        const double sv = s[2 * dof + c], ev = xstar[2 * dof + c] - x[2 * dof + c];
        in_img[(patch * 2 + c) * per + pix] = (float)(sv * inv);
        tgt_img[(patch * 2 + c) * per + pix] = (float)((ev - sv) * inv);
    }
}

}  // namespace

ibem_status solver_pairs_impl(ibem_handle* h, const double* b, int nrhs, double rtol, int maxit, int stride,
                              int max_pairs, float* in_img, float* tgt_img, int* n_pairs, ibem_solve_info* info) {
    Plan& P = h->P;
    const int64_t N = P.N;
    cudaStream_t st = h->stream;
    auto t0 = std::chrono::steady_clock::now();
    const size_t vec = (size_t)2 * N;
    double *X = nullptr, *R = nullptr, *xs = nullptr, *s = nullptr;
    auto release = [&](ibem_status r) {
        if (X) cudaFreeAsync(X, st);
        if (R) cudaFreeAsync(R, st);
        if (xs) cudaFreeAsync(xs, st);
        if (s) cudaFreeAsync(s, st);
        cudaStreamSynchronize(st);
        return r;
    };
    if (cudaMallocAsync(&X, (size_t)max_pairs * vec * sizeof(double), st) ||
        cudaMallocAsync(&R, (size_t)max_pairs * vec * sizeof(double), st) ||
        cudaMallocAsync(&xs, vec * sizeof(double), st) || cudaMallocAsync(&s, vec * sizeof(double), st))
        return release(IBEM_ERR_OOM);
    const size_t img = (size_t)P.npatch * 2 * P.n1 * P.n1;
    int total = 0, total_it = 0, total_outer = 0;
    double worst = 0.0;
    ibem_status worst_s = IBEM_OK;
    for (int r = 0; r < nrhs; ++r) {
        const double* bb = b + (size_t)r * vec;
        double nb;
        if (norm2(h, bb, vec, &nb) != cudaSuccess) return release(IBEM_ERR_CUDA);
        if (nb == 0.0) continue;
        Recorder rec;
        rec.stride = stride;
        rec.max = max_pairs;
        rec.X = X;
        rec.R = R;
        int its = 0, outer = 0;
        ibem_status sres = gmres(h, bb, xs, rtol * nb, maxit, IBEM_PRECOND_BLOCK_JACOBI, IBEM_FP64,
                                 std::max(100, std::min(maxit, 400)), &its, &outer, &rec);
        if (sres != IBEM_OK && sres != IBEM_ERR_NOCONV) return release(sres);
        if (sres != IBEM_OK && worst_s == IBEM_OK) worst_s = sres;
        // true residual of x*
        if (apply_operator(h, xs, s, 1, IBEM_FP64) != cudaSuccess) return release(IBEM_ERR_CUDA);
        sub_kernel<<<nblk(vec, 256), 256, 0, st>>>(vec, bb, s, s);
        double rt;
        if (norm2(h, s, vec, &rt) != cudaSuccess) return release(IBEM_ERR_CUDA);
        worst = std::max(worst, rt / nb);
        total_it += its;
        total_outer += outer;
        for (int n = 0; n < rec.n; ++n) {
            apply_block_jacobi(h, R + (size_t)n * vec, s);
            dot_kernel<<<1, 1024, 0, st>>>(s, s, vec, h->d_red);
            pair_images_kernel<<<nblk(N, 256), 256, 0, st>>>(N, P.n1, xs, X + (size_t)n * vec, s, h->d_red,
                                                             in_img + (size_t)(total + n) * img,
                                                             tgt_img + (size_t)(total + n) * img);
        }
        total += rec.n;
    }
    if (cudaGetLastError() != cudaSuccess) return release(IBEM_ERR_CUDA);
    *n_pairs = total;
    if (info) {
        info->iterations = total_it;
        info->outer = total_outer;
        info->rel_residual = worst;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->steps = total_it;
    }
    return release(worst_s);
}

// dst = src / sqrt(nrm2[0]) (zero if nrm2[0] = 0)
__global__ void normalize_copy_kernel(int64_t n, const double* __restrict__ src, const double* __restrict__ nrm2,
                                      double* __restrict__ dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dst[i] = nrm2[0] > 0.0 ? src[i] / sqrt(nrm2[0]) : 0.0;
}

ibem_status solver_residuals_impl(ibem_handle* h, const double* b, int nrhs, double rtol, int maxit, int stride,
                                  int max_vecs, double* r_out, int* n_out, ibem_solve_info* info) {
    Plan& P = h->P;
    const int64_t N = P.N;
    cudaStream_t st = h->stream;
    auto t0 = std::chrono::steady_clock::now();
    const size_t vec = (size_t)2 * N;
    double *R = nullptr, *xs = nullptr;
    auto release = [&](ibem_status r) {
        if (R) cudaFreeAsync(R, st);
        if (xs) cudaFreeAsync(xs, st);
        cudaStreamSynchronize(st);
        return r;
    };
    if (cudaMallocAsync(&R, (size_t)max_vecs * vec * sizeof(double), st) ||
        cudaMallocAsync(&xs, vec * sizeof(double), st))
        return release(IBEM_ERR_OOM);
    int total = 0, total_it = 0, total_outer = 0;
    ibem_status worst_s = IBEM_OK;
    for (int r = 0; r < nrhs; ++r) {
        const double* bb = b + (size_t)r * vec;
        double nb;
        if (norm2(h, bb, vec, &nb) != cudaSuccess) return release(IBEM_ERR_CUDA);
        if (nb == 0.0) continue;
        Recorder rec;
        rec.stride = stride;
        rec.max = max_vecs;
        rec.R = R;
        int its = 0, outer = 0;
        ibem_status sres = gmres(h, bb, xs, rtol * nb, maxit, IBEM_PRECOND_BLOCK_JACOBI, IBEM_FP64,
                                 std::max(100, std::min(maxit, 400)), &its, &outer, &rec);
        if (sres != IBEM_OK && sres != IBEM_ERR_NOCONV) return release(sres);
        if (sres != IBEM_OK && worst_s == IBEM_OK) worst_s = sres;
        total_it += its;
        total_outer += outer;
        for (int n = 0; n < rec.n; ++n) {
            dot_kernel<<<1, 1024, 0, st>>>(R + (size_t)n * vec, R + (size_t)n * vec, vec, h->d_red);
            normalize_copy_kernel<<<nblk(vec, 256), 256, 0, st>>>(vec, R + (size_t)n * vec, h->d_red,
                                                                  r_out + (size_t)(total + n) * vec);
        }
        total += rec.n;
    }
    if (cudaGetLastError() != cudaSuccess) return release(IBEM_ERR_CUDA);
    *n_out = total;
    if (info) {
        info->iterations = total_it;
        info->outer = total_outer;
        info->rel_residual = 0.0;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->steps = total_it;
    }
    return release(worst_s);
}

ibem_status solve_impl(ibem_handle* h, const double* b, double* wout, int nrhs, double rtol, int maxit,
                       int precond, int precision, ibem_solve_info* info) {
    if (nrhs > 1) return solve_block_impl(h, b, wout, nrhs, rtol, maxit, precond, precision, info);
    Plan& P = h->P;
    int64_t N = P.N;
    auto t0 = std::chrono::steady_clock::now();
    size_t need = 7 * (size_t)N * (h->helm ? 2 : 1);
    if (h->solver_len < need) {
        cudaFree(h->d_solver);
        h->d_solver = nullptr;
        h->solver_len = 0;
        if (cudaMalloc(&h->d_solver, need * sizeof(double)) != cudaSuccess) return IBEM_ERR_OOM;
        h->solver_len = need;
    }
    const int64_t NN = N * (h->helm ? 2 : 1);
    Work w{h->d_solver, h->d_solver + NN, h->d_solver + 2 * NN, h->d_solver + 3 * NN, h->d_solver + 4 * NN,
           h->d_solver + 5 * NN, h->d_solver + 6 * NN};

    ibem_status worst = IBEM_OK;
    int total_it = 0, total_outer = 0;
    double worst_res = 0.0;
    cudaStream_t st = h->stream;
    for (int rhs = 0; rhs < nrhs; ++rhs) {
        const int cw = h->helm ? 2 : 1;            // doubles per entry
        const double* bb = b + (size_t)rhs * N * cw;
        double* ww = wout + (size_t)rhs * N * cw;
        double nb;
        if (norm2(h, bb, cw * N, &nb) != cudaSuccess) return IBEM_ERR_CUDA;
        if (nb == 0.0) {
            cudaMemsetAsync(ww, 0, cw * N * sizeof(double), st);
            continue;
        }
        ibem_status s = IBEM_OK;
        int its = 0, outer = 0;
        double res = 0.0;
        if (h->helm) {
            s = gmres(h, bb, ww, rtol * nb, maxit, precond, precision, 100, &its, &outer);
        } else if (precision == IBEM_FP64) {
            s = cg(h, bb, ww, w, IBEM_FP64, rtol * nb, maxit, precond, &its);
            outer = 1;
        } else {
            s = cg_reliable(h, bb, ww, w, rtol * nb, maxit, precond, &its, &outer);
        }
        // true residual with the FP64 operator
        if (apply_operator(h, ww, w.Ap, 1, IBEM_FP64) != cudaSuccess) return IBEM_ERR_CUDA;
        sub_kernel<<<nblk(cw * N, 256), 256, 0, st>>>(cw * N, bb, w.Ap, w.rr);
        double rt;
        if (norm2(h, w.rr, cw * N, &rt) != cudaSuccess) return IBEM_ERR_CUDA;
        res = rt / nb;
        if (s == IBEM_OK && res > rtol * 1.0001) s = IBEM_ERR_NOCONV;
        total_it += its;
        total_outer += outer;
        if (res > worst_res) worst_res = res;
        if (s != IBEM_OK && worst == IBEM_OK) worst = s;
    }
    if (info) {
        info->iterations = total_it;
        info->outer = total_outer;
        info->rel_residual = worst_res;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->steps = total_it;
    }
    return worst;
}

}  // namespace ibem
