// Solving every instance of a batch (Sec. 4 item 3 for many uneven problems):
// lock-step restarted GMRES over all columns (instance, right-hand side) of the
// concatenated arrays, each column with its own Krylov space and stopping test,
// where one step applies the batched FP32 operator (one graph launch for all
// instances).  Outer loop: the residual r = b - A x of every column with each
// instance's FP64 operator when every handle has one (iterative refinement:
// the inner cycles stop at max(rtol |b|, 1e-3 |r|)), else with the batched FP32
// operator itself (the inner cycles then aim at rtol |b|); converged columns
// keep their solution and take zero basis vectors.  Laplace and Helmholtz
// columns share the GMRES code (real columns have zero imaginary parts).
//
// Columns are segments of the flat vector: column c starts at off[c] doubles,
// holds n[c] entries of cw[c] doubles.  Reductions are one CTA per (basis
// vector, column) with a fixed tree: deterministic.
#include <chrono>
#include <cmath>

#include "batch_internal.cuh"
#include "gmres_column.h"

namespace ibem {
namespace {

struct SegCol {
    int64_t off, n;
    int cw;
};

inline unsigned sblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// column of entry e: the last c with eoff[c] <= e
__device__ inline int seg_find(const int64_t* __restrict__ eoff, int ncol, int64_t e) {
    int lo = 0, hi = ncol;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (eoff[mid] <= e) lo = mid;
        else hi = mid;
    }
    return lo;
}

// out[k][c] = sum_i conj(V_k[c][i]) w[c][i]; grid (nk, ncol)
__global__ void seg_dots_kernel(const double* __restrict__ V, int64_t T, const SegCol* __restrict__ cols,
                                const double* __restrict__ w, int ncol, double* __restrict__ out) {
    __shared__ double sr[256], si[256];
    const int k = blockIdx.x, c = blockIdx.y;
    const SegCol C = cols[c];
    const double* v = V + (int64_t)k * T + C.off;
    const double* x = w + C.off;
    double ar = 0.0, ai = 0.0;
    for (int64_t i = threadIdx.x; i < C.n; i += blockDim.x) {
        if (C.cw == 1) {
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
        out[2 * ((int64_t)k * ncol + c)] = sr[0];
        out[2 * ((int64_t)k * ncol + c) + 1] = si[0];
    }
}

// out[c] = |x[c]|^2; grid ncol
__global__ void seg_norm2_kernel(const double* __restrict__ x, const SegCol* __restrict__ cols,
                                 double* __restrict__ out) {
    __shared__ double s[256];
    const SegCol C = cols[blockIdx.x];
    const double* v = x + C.off;
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < C.n * C.cw; i += blockDim.x) a += v[i] * v[i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

// mode 0: w -= sum_{k < nk} V_k h[k]; mode 1: out = sum_{k < nk} V_k h[k];
// mode 2: out = h[0] w (real scale per column, h[c]).  Flat over entries.
__global__ void seg_combine_kernel(int mode, const double* __restrict__ V, int64_t T, int nk,
                                   const SegCol* __restrict__ cols, const int64_t* __restrict__ eoff, int ncol,
                                   int64_t nent, const double* __restrict__ h, double* __restrict__ w,
                                   double* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nent) return;
    const int c = seg_find(eoff, ncol, e);
    const SegCol C = cols[c];
    const int64_t d = C.off + (e - eoff[c]) * C.cw;
    if (mode == 2) {
        const double s = h[c];
        out[d] = s * w[d];
        if (C.cw == 2) out[d + 1] = s * w[d + 1];
        return;
    }
    double ar = 0.0, ai = 0.0;
    for (int k = 0; k < nk; ++k) {
        const double hr = h[2 * ((int64_t)k * ncol + c)], hi = h[2 * ((int64_t)k * ncol + c) + 1];
        const double* v = V + (int64_t)k * T + d;
        if (C.cw == 1) {
            ar += v[0] * hr;
        } else {
            ar += v[0] * hr - v[1] * hi;
            ai += v[0] * hi + v[1] * hr;
        }
    }
    if (mode == 0) {
        w[d] -= ar;
        if (C.cw == 2) w[d + 1] -= ai;
    } else {
        out[d] = ar;
        if (C.cw == 2) out[d + 1] = ai;
    }
}

__global__ void flat_axpy_kernel(int64_t n, double a, const double* __restrict__ x, const double* __restrict__ y,
                                 double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = y[i] + a * x[i];
}

// z = v / d for R columns of n entries (complex division if cw = 2; d null: copy)
__global__ void inst_jacobi_kernel(const double* __restrict__ v, const double* __restrict__ d, int64_t n, int R,
                                   int cw, double* __restrict__ z) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)R * n) return;
    const int64_t i = idx % n;
    if (cw == 1) {
        z[idx] = d ? v[idx] / d[i] : v[idx];
    } else if (d) {
        const double vr = v[2 * idx], vi = v[2 * idx + 1], dr = d[2 * i], di = d[2 * i + 1], den = dr * dr + di * di;
        z[2 * idx] = (vr * dr + vi * di) / den;
        z[2 * idx + 1] = (vi * dr - vr * di) / den;
    } else {
        z[2 * idx] = v[2 * idx];
        z[2 * idx + 1] = v[2 * idx + 1];
    }
}

struct BatchKrylov {
    ibem_batch* b;
    cudaStream_t st;
    int ncol = 0;
    int64_t T = 0, nent = 0;
    std::vector<SegCol> cols;
    std::vector<int> col_inst, col_r;
    SegCol* d_cols = nullptr;
    int64_t* d_eoff = nullptr;
    double* d_red = nullptr;
    double* h_red = nullptr;
    size_t red = 0;
    int precond = IBEM_PRECOND_JACOBI;
    bool fp64 = false;
    std::vector<cudaStream_t> saved;
    std::vector<void*> owned;

    ~BatchKrylov() {
        for (size_t i = 0; i < saved.size(); ++i) b->handles[i]->stream = saved[i];
        for (void* p : owned) cudaFree(p);
        if (h_red) cudaFreeHost(h_red);
    }
    template <typename X>
    bool alloc(X** p, size_t count) {
        if (cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(X) + 16) != cudaSuccess) return false;
        owned.push_back(*p);
        return true;
    }
    cudaError_t read(size_t count, std::vector<double>& out) {
        cudaError_t e;
        if ((e = cudaMemcpyAsync(h_red, d_red, count * sizeof(double), cudaMemcpyDeviceToHost, st))) return e;
        if ((e = cudaStreamSynchronize(st))) return e;
        out.assign(h_red, h_red + count);
        return cudaSuccess;
    }
    cudaError_t upload(const std::vector<double>& v, double* dst) {
        std::copy(v.begin(), v.end(), h_red + red);
        cudaError_t e = cudaMemcpyAsync(dst, h_red + red, v.size() * sizeof(double), cudaMemcpyHostToDevice, st);
        return e ? e : cudaStreamSynchronize(st);
    }
    cudaError_t norms(const double* x, std::vector<double>& out) {
        seg_norm2_kernel<<<ncol, 256, 0, st>>>(x, d_cols, d_red);
        cudaError_t e = read(ncol, out);
        for (double& v : out) v = std::sqrt(v);
        return e;
    }
    // y = A x with the batched FP32 operator (fixed input and output buffers, so
    // the captured graph is replayed)
    cudaError_t apply32(const double* x, double* y) {
        cudaError_t e;
        if ((e = cudaMemcpyAsync(b->solve_x, x, T * sizeof(double), cudaMemcpyDeviceToDevice, st))) return e;
        if (ibem_batch_matvec(b, b->solve_x, b->solve_y) != IBEM_OK) return cudaErrorUnknown;
        return cudaMemcpyAsync(y, b->solve_y, T * sizeof(double), cudaMemcpyDeviceToDevice, st);
    }
    // y = A x with every instance's FP64 operator (on the batch stream)
    cudaError_t apply64(const double* x, double* y) {
        for (int i = 0; i < b->n; ++i) {
            cudaError_t e = apply_operator(b->handles[i], x + b->offsets[i], y + b->offsets[i], b->inst[i].R, IBEM_FP64);
            if (e) return e;
        }
        return cudaGetLastError();
    }
    cudaError_t precondition(const double* v, double* z) {
        for (int i = 0; i < b->n; ++i) {
            ibem_handle* h = b->handles[i];
            const BatchInst& I = b->inst[i];
            const int cw = I.helm ? 2 : 1;
            if (precond == IBEM_PRECOND_BLOCK_JACOBI) {
                for (int r = 0; r < I.R; ++r)
                    apply_block_jacobi(h, v + b->offsets[i] + (int64_t)r * I.N * cw,
                                       z + b->offsets[i] + (int64_t)r * I.N * cw);
            } else {
                inst_jacobi_kernel<<<sblk((int64_t)I.R * I.N, 256), 256, 0, st>>>(
                    v + b->offsets[i], precond == IBEM_PRECOND_JACOBI ? h->d_diag : nullptr, I.N, I.R, cw,
                    z + b->offsets[i]);
            }
        }
        return cudaGetLastError();
    }
};

}  // namespace
}  // namespace ibem

using namespace ibem;

extern "C" ibem_status ibem_batch_solve(ibem_batch* b, const double* b_dev, double* x_dev, double rtol, int maxit,
                                        int precond, ibem_solve_info* info) {
    if (!b || !b_dev || !x_dev || !(rtol > 0.0) || maxit < 1) return IBEM_ERR_ARG;
    if (precond != IBEM_PRECOND_NONE && precond != IBEM_PRECOND_JACOBI && precond != IBEM_PRECOND_BLOCK_JACOBI)
        return IBEM_ERR_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return IBEM_ERR_CUDA;
    auto t0 = std::chrono::steady_clock::now();
    const int restart = 100;
    BatchKrylov K;
    K.b = b;
    K.st = b->stream;
    K.precond = precond;
    // every instance-level operation of the solve runs on the batch stream
    for (ibem_handle* h : b->handles) {
        K.saved.push_back(h->stream);
        h->stream = b->stream;
    }
    K.fp64 = true;
    for (ibem_handle* h : b->handles)
        if (!h->d_near || (!h->helm && h->P.q > 0 && !h->far_rows.empty() && !h->d_K && !h->d_Kdf)) K.fp64 = false;
    std::vector<int64_t> eoff;
    for (int i = 0; i < b->n; ++i) {
        const BatchInst& I = b->inst[i];
        const int cw = I.helm ? 2 : 1;
        for (int r = 0; r < I.R; ++r) {
            eoff.push_back(K.nent);
            K.cols.push_back({b->offsets[i] + (int64_t)r * I.N * cw, I.N, cw});
            K.col_inst.push_back(i);
            K.col_r.push_back(r);
            K.nent += I.N;
        }
    }
    K.ncol = (int)K.cols.size();
    K.T = b->offsets[b->n];
    const int nc = K.ncol;
    const int64_t T = K.T;
    K.red = (size_t)6 * (restart + 2) * nc + 64;
    if (cudaMallocHost(&K.h_red, 2 * K.red * sizeof(double)) != cudaSuccess) return IBEM_ERR_OOM;
    double *V = nullptr, *w = nullptr, *tmp = nullptr, *r = nullptr, *d = nullptr, *dh = nullptr;
    if (!K.alloc(&K.d_cols, nc) || !K.alloc(&K.d_eoff, nc) || !K.alloc(&K.d_red, K.red) ||
        !K.alloc(&V, (size_t)(restart + 1) * T) || !K.alloc(&w, T) || !K.alloc(&tmp, T) || !K.alloc(&r, T) ||
        !K.alloc(&d, T) || !K.alloc(&dh, (size_t)6 * (restart + 2) * nc))
        return IBEM_ERR_OOM;
    if (!b->solve_x && (cudaMalloc(&b->solve_x, T * sizeof(double)) || cudaMalloc(&b->solve_y, T * sizeof(double))))
        return IBEM_ERR_OOM;
    cudaStream_t st = K.st;
    if (cudaMemcpyAsync(K.d_cols, K.cols.data(), nc * sizeof(SegCol), cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(K.d_eoff, eoff.data(), nc * sizeof(int64_t), cudaMemcpyHostToDevice, st))
        return IBEM_ERR_CUDA;
    const unsigned gT = sblk(T, 256), gE = sblk(K.nent, 256);
    std::vector<double> nb, rn;
    if (K.norms(b_dev, nb) != cudaSuccess) return IBEM_ERR_CUDA;
    for (double v : nb)
        if (!std::isfinite(v)) return IBEM_ERR_BREAKDOWN;   // NaN or Inf in the right-hand sides
    cudaMemsetAsync(x_dev, 0, T * sizeof(double), st);
    cudaMemcpyAsync(r, b_dev, T * sizeof(double), cudaMemcpyDeviceToDevice, st);
    const double delta = K.fp64 ? 1e-3 : 0.0;
    int steps = 0, outer = 0, total_its = 0;
    ibem_status status = IBEM_OK;
    for (;;) {
        if (K.norms(r, rn) != cudaSuccess) return IBEM_ERR_CUDA;
        std::vector<char> active(nc, 0);
        std::vector<double> tol(nc, 0.0), scale(nc, 0.0);
        int nact = 0;
        for (int c = 0; c < nc; ++c) {
            if (!std::isfinite(rn[c])) return IBEM_ERR_BREAKDOWN;
            if (rn[c] > rtol * nb[c]) {
                active[c] = 1;
                ++nact;
                tol[c] = std::max(rtol * nb[c], delta * rn[c]);
                scale[c] = 1.0 / rn[c];
            }
        }
        if (nact == 0) break;
        if (steps >= maxit) {
            status = IBEM_ERR_NOCONV;
            break;
        }
        ++outer;
        // one GMRES(restart) cycle from x0 = 0 on A d = r
        if (K.upload(scale, K.d_red) != cudaSuccess) return IBEM_ERR_CUDA;
        seg_combine_kernel<<<gE, 256, 0, st>>>(2, nullptr, T, 0, K.d_cols, K.d_eoff, nc, K.nent, K.d_red, r, V);
        std::vector<GmresColumn> col(nc);
        for (int c = 0; c < nc; ++c) col[c].start(restart, active[c] ? rn[c] : 0.0);
        int j = 0;
        std::vector<double> hb, hq;
        for (; j < restart && nact > 0 && steps < maxit; ++j) {
            double* Vj = V + (size_t)j * T;
            if (K.precondition(Vj, tmp) != cudaSuccess || K.apply32(tmp, w) != cudaSuccess) return IBEM_ERR_CUDA;
            ++steps;
            double* h0 = dh;
            double* h1 = dh + (size_t)2 * (j + 1) * nc;
            double* hn = dh + (size_t)4 * (j + 1) * nc;
            for (int pass = 0; pass < 2; ++pass) {
                double* hp = pass == 0 ? h0 : h1;
                seg_dots_kernel<<<dim3(j + 1, nc), 256, 0, st>>>(V, T, K.d_cols, w, nc, hp);
                seg_combine_kernel<<<gE, 256, 0, st>>>(0, V, T, j + 1, K.d_cols, K.d_eoff, nc, K.nent, hp, w,
                                                       nullptr);
            }
            seg_norm2_kernel<<<nc, 256, 0, st>>>(w, K.d_cols, hn);
            if (cudaMemcpyAsync(K.h_red, dh, ((size_t)4 * (j + 1) * nc + nc) * sizeof(double),
                                cudaMemcpyDeviceToHost, st) ||
                cudaStreamSynchronize(st))
                return IBEM_ERR_CUDA;
            hb.assign(K.h_red, K.h_red + (size_t)4 * (j + 1) * nc + nc);
            for (int c = 0; c < nc; ++c) {
                scale[c] = 0.0;
                if (!active[c]) continue;
                hq.assign(2 * (j + 1), 0.0);
                for (int i = 0; i <= j; ++i) {
                    hq[2 * i] = hb[2 * ((size_t)i * nc + c)] + hb[(size_t)2 * (j + 1) * nc + 2 * ((size_t)i * nc + c)];
                    hq[2 * i + 1] = hb[2 * ((size_t)i * nc + c) + 1] +
                                    hb[(size_t)2 * (j + 1) * nc + 2 * ((size_t)i * nc + c) + 1];
                }
                const double hnc = std::sqrt(hb[(size_t)4 * (j + 1) * nc + c]);
                const double res = col[c].add(j, hq.data(), hnc);
                if (res < 0.0 || !std::isfinite(hnc)) return IBEM_ERR_BREAKDOWN;
                ++total_its;
                if (res <= tol[c] || hnc == 0.0) {
                    active[c] = 0;
                    --nact;
                } else {
                    scale[c] = 1.0 / hnc;
                }
            }
            if (K.upload(scale, K.d_red) != cudaSuccess) return IBEM_ERR_CUDA;
            seg_combine_kernel<<<gE, 256, 0, st>>>(2, nullptr, T, 0, K.d_cols, K.d_eoff, nc, K.nent, K.d_red, w,
                                                   V + (size_t)(j + 1) * T);
        }
        if (j > 0) {
            std::vector<double> y((size_t)2 * j * nc, 0.0), yy;
            for (int c = 0; c < nc; ++c) {
                col[c].solve(yy);
                for (int i = 0; i < col[c].k; ++i) {
                    y[2 * ((size_t)i * nc + c)] = yy[2 * i];
                    y[2 * ((size_t)i * nc + c) + 1] = yy[2 * i + 1];
                }
            }
            if (K.upload(y, dh) != cudaSuccess) return IBEM_ERR_CUDA;
            seg_combine_kernel<<<gE, 256, 0, st>>>(1, V, T, j, K.d_cols, K.d_eoff, nc, K.nent, dh, nullptr, w);
            if (K.precondition(w, d) != cudaSuccess) return IBEM_ERR_CUDA;
            flat_axpy_kernel<<<gT, 256, 0, st>>>(T, 1.0, d, x_dev, x_dev);
        }
        // r = b - A x (FP64 operators of the instances, else the batched FP32 one)
        if ((K.fp64 ? K.apply64(x_dev, w) : K.apply32(x_dev, w)) != cudaSuccess) return IBEM_ERR_CUDA;
        flat_axpy_kernel<<<gT, 256, 0, st>>>(T, -1.0, w, b_dev, r);
    }
    double worst = 0.0;
    if (K.norms(r, rn) != cudaSuccess) return IBEM_ERR_CUDA;
    for (int c = 0; c < nc; ++c)
        if (nb[c] > 0.0) worst = std::max(worst, rn[c] / nb[c]);
    if (info) {
        info->iterations = total_its;
        info->outer = outer;
        info->rel_residual = worst;
        info->steps = steps;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    cudaStreamSynchronize(st);
    return status;
}
