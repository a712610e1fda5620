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
               int maxit, bool jacobi, int* its) {
    Plan& P = h->P;
    int64_t N = P.N;
    cudaStream_t st = h->stream;
    const double* d = jacobi ? h->d_diag : nullptr;
    cudaMemsetAsync(x, 0, N * sizeof(double), st);
    cudaMemcpyAsync(w.r, b, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    scal_div_kernel<<<nblk(N, 256), 256, 0, st>>>(N, w.r, d, w.z);
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
                        bool jacobi, int* its, int* updates) {
    Plan& P = h->P;
    int64_t N = P.N;
    cudaStream_t st = h->stream;
    const double* d = jacobi ? h->d_diag : nullptr;
    const double drop = 1e-2;
    cudaMemsetAsync(x, 0, N * sizeof(double), st);
    cudaMemcpyAsync(w.r, b, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    scal_div_kernel<<<nblk(N, 256), 256, 0, st>>>(N, w.r, d, w.z);
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
            dot_kernel<<<1, 1024, 0, st>>>(w.r, w.z, N, h->d_red);
            if (readback(h, h->d_red, 1, &rz_new) != cudaSuccess) return IBEM_ERR_CUDA;
        }
        double beta = rz_new / rz;
        rz = rz_new;
        xpby_kernel<<<nblk(N, 256), 256, 0, st>>>(N, w.z, beta, w.p);
    }
    return IBEM_ERR_NOCONV;
}

}  // namespace

ibem_status solve_impl(ibem_handle* h, const double* b, double* wout, int nrhs, double rtol, int maxit,
                       int precond, int precision, ibem_solve_info* info) {
    Plan& P = h->P;
    int64_t N = P.N;
    auto t0 = std::chrono::steady_clock::now();
    size_t need = 7 * (size_t)N;
    if (h->solver_len < need) {
        cudaFree(h->d_solver);
        h->d_solver = nullptr;
        h->solver_len = 0;
        if (cudaMalloc(&h->d_solver, need * sizeof(double)) != cudaSuccess) return IBEM_ERR_OOM;
        h->solver_len = need;
    }
    Work w{h->d_solver, h->d_solver + N, h->d_solver + 2 * N, h->d_solver + 3 * N, h->d_solver + 4 * N,
           h->d_solver + 5 * N, h->d_solver + 6 * N};
    bool jac = precond == IBEM_PRECOND_JACOBI;
    ibem_status worst = IBEM_OK;
    int total_it = 0, total_outer = 0;
    double worst_res = 0.0;
    cudaStream_t st = h->stream;
    for (int rhs = 0; rhs < nrhs; ++rhs) {
        const double* bb = b + (size_t)rhs * N;
        double* ww = wout + (size_t)rhs * N;
        double nb;
        if (norm2(h, bb, N, &nb) != cudaSuccess) return IBEM_ERR_CUDA;
        if (nb == 0.0) {
            cudaMemsetAsync(ww, 0, N * sizeof(double), st);
            continue;
        }
        ibem_status s = IBEM_OK;
        int its = 0, outer = 0;
        double res = 0.0;
        if (precision == IBEM_FP64) {
            s = cg(h, bb, ww, w, IBEM_FP64, rtol * nb, maxit, jac, &its);
            outer = 1;
        } else {
            s = cg_reliable(h, bb, ww, w, rtol * nb, maxit, jac, &its, &outer);
        }
        // true residual with the FP64 operator
        if (apply_operator(h, ww, w.Ap, 1, IBEM_FP64) != cudaSuccess) return IBEM_ERR_CUDA;
        sub_kernel<<<nblk(N, 256), 256, 0, st>>>(N, bb, w.Ap, w.rr);
        double rt;
        if (norm2(h, w.rr, N, &rt) != cudaSuccess) return IBEM_ERR_CUDA;
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
    }
    return worst;
}

}  // namespace ibem
