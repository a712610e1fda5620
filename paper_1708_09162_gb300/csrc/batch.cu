// Batched application of many uneven problem instances (FP32 operator).
//
// A batch holds assembled handles of different sizes (level, degree, kernel,
// number of right-hand sides).  One application runs every stage of the
// operator - T^T, leaf moments, M2M per level, coupling, L2L per level,
// back-projection, near field, T - as ONE launch per stage over a flat work list
// that spans all instances (each thread finds its instance by binary search in a
// prefix table).  The far-field coupling is a persistent kernel: as many CTAs as
// fit on the GPU take (instance, right-hand side, target cluster) items from an
// atomic counter, so uneven instances balance dynamically.  The whole
// application (about 2 max(m) + 8 launches, independent of the number of
// instances) is captured once into a CUDA graph and replayed.  The CTA size of
// the coupling kernel is chosen at batch creation by timing the candidates
// (autotuning).
//
// Per instance the FP32 work vectors live in one arena: x* [R][E][nb][cw],
// x^ and y^ [R][C][q2][cw], y* [R][E][nb][cw] with cw = 1 (Laplace) or 2
// (Helmholtz, interleaved).  Inputs and outputs are the caller's concatenated
// FP64 arrays (instance i at offsets[i], [R_i][N_i] values, complex interleaved).
#include <algorithm>
#include <chrono>
#include <cstring>

#include "batch_internal.cuh"

namespace ibem {

static inline unsigned bblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ inline int find_inst(const int64_t* __restrict__ pre, int n, int64_t g) {
    int lo = 0, hi = n;   // pre[lo] <= g < pre[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (pre[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ inline void inst_elem(const BatchInst& I, int64_t e, int* patch, int* ix, int* iy) {
    int64_t per = (int64_t)I.ne1 * I.ne1;
    *patch = (int)(e / per);
    uint32_t x, y;
    morton2_inv((uint32_t)(e % per), &x, &y);
    *ix = (int)x;
    *iy = (int)y;
}

// x* = T^T x; item (r, e, i)
__global__ void b_lift_kernel(const BatchInst* __restrict__ B, int n, const int64_t* __restrict__ pre, int64_t total,
                              const double* __restrict__ x) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int k = find_inst(pre, n, g);
    const BatchInst& I = B[k];
    int64_t loc = g - pre[k];
    const int i = (int)(loc % I.nb);
    loc /= I.nb;
    const int64_t e = loc % I.E;
    const int r = (int)(loc / I.E);
    int patch, ix, iy;
    inst_elem(I, e, &patch, &ix, &iy);
    const int iu = i % I.pp, iv = i / I.pp, cw = I.helm ? 2 : 1;
    float ar = 0.0f, ai = 0.0f;
    const double* xr = x + I.xoff + (int64_t)r * I.N * cw;
    for (int r2 = 0; r2 < I.pp; ++r2)
        for (int r1 = 0; r1 < I.pp; ++r1) {
            const float c = (float)I.ext[((int64_t)iy * I.pp + r2) * I.pp + iv] *
                            (float)I.ext[((int64_t)ix * I.pp + r1) * I.pp + iu];
            const int64_t dof = (int64_t)patch * I.n1 * I.n1 + (int64_t)(iy + r2) * I.n1 + (ix + r1);
            ar = fmaf(c, (float)xr[dof * cw], ar);
            if (cw == 2) ai = fmaf(c, (float)xr[dof * 2 + 1], ai);
        }
    float* o = I.xs + (((int64_t)r * I.E + e) * I.nb + i) * cw;
    o[0] = ar;
    if (cw == 2) o[1] = ai;
}

// leaf moments; item (r, e, a)
__global__ void b_leaf_kernel(const BatchInst* __restrict__ B, int n, const int64_t* __restrict__ pre, int64_t total) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int k = find_inst(pre, n, g);
    const BatchInst& I = B[k];
    int64_t loc = g - pre[k];
    const int a = (int)(loc % I.q2);
    loc /= I.q2;
    const int64_t e = loc % I.E;
    const int r = (int)(loc / I.E);
    const int au = a % I.q, av = a / I.q, cw = I.helm ? 2 : 1;
    float ar = 0.0f, ai = 0.0f;
    const float* v = I.xs + ((int64_t)r * I.E + e) * I.nb * cw;
    for (int iv = 0; iv < I.pp; ++iv)
        for (int iu = 0; iu < I.pp; ++iu) {
            const float c = I.Mf[au * I.pp + iu] * I.Mf[av * I.pp + iv];
            ar = fmaf(c, v[(iv * I.pp + iu) * cw], ar);
            if (cw == 2) ai = fmaf(c, v[(iv * I.pp + iu) * 2 + 1], ai);
        }
    float* o = I.xh + (((int64_t)r * I.C + I.lvl[I.m] + e) * I.q2 + a) * cw;
    o[0] = ar;
    if (cw == 2) o[1] = ai;
}

// M2M for parents at level m - kk of every instance with m >= kk; item (r, pl, a)
__global__ void b_m2m_kernel(const BatchInst* __restrict__ B, int n, const int64_t* __restrict__ pre, int64_t total,
                             int kk) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int k = find_inst(pre, n, g);
    const BatchInst& I = B[k];
    const int L = I.m - kk;
    const int64_t nL = I.lvl[L + 1] - I.lvl[L];
    int64_t loc = g - pre[k];
    const int a = (int)(loc % I.q2);
    loc /= I.q2;
    const int64_t pl = loc % nL;
    const int r = (int)(loc / nL);
    const int q = I.q, q2 = I.q2, au = a % q, av = a / q, cw = I.helm ? 2 : 1;
    float ar = 0.0f, ai = 0.0f;
    for (int c = 0; c < 4; ++c) {
        const float* Su = I.Sf + (c & 1) * q2;
        const float* Sv = I.Sf + (c >> 1) * q2;
        const float* v = I.xh + (((int64_t)r * I.C + I.lvl[L + 1] + 4 * pl + c) * q2) * cw;
        for (int bv = 0; bv < q; ++bv) {
            float tr = 0.0f, ti = 0.0f;
            for (int bu = 0; bu < q; ++bu) {
                tr = fmaf(Su[au * q + bu], v[(bv * q + bu) * cw], tr);
                if (cw == 2) ti = fmaf(Su[au * q + bu], v[(bv * q + bu) * 2 + 1], ti);
            }
            ar = fmaf(Sv[av * q + bv], tr, ar);
            ai = fmaf(Sv[av * q + bv], ti, ai);
        }
    }
    float* o = I.xh + (((int64_t)r * I.C + I.lvl[L] + pl) * q2 + a) * cw;
    o[0] = ar;
    if (cw == 2) o[1] = ai;
}

// Persistent coupling: CTAs take (instance, r, row) items from *counter.
// Thread t = g * q2 + a (g < G = blockDim / q2) sums target point a against the
// blocks g, g + G, ... of the row; partial sums meet in shared memory.
// Right-hand sides per coupling work item: every kernel value generated for a
// far block serves up to RB right-hand sides of the instance (the tile shape
// chosen with the CTA size by the autotuner: RB in 4, 8, 16).

template <int BC_RB>
__global__ void b_coupling_kernel(const BatchInst* __restrict__ B, int n, const int64_t* __restrict__ pre,
                                  int64_t total, int* __restrict__ counter) {
    extern __shared__ float red[];   // [BC_RB][blockDim][2]
    __shared__ int64_t item;
    for (;;) {
        if (threadIdx.x == 0) item = atomicAdd(counter, 1);
        __syncthreads();
        const int64_t it = item;
        if (it >= total) break;
        const int k = find_inst(pre, n, it);
        const BatchInst& I = B[k];
        const int64_t loc = it - pre[k];
        const int nch = (I.R + BC_RB - 1) / BC_RB;
        const int64_t nrows = (pre[k + 1] - pre[k]) / nch;
        const int r0 = (int)(loc / nrows) * BC_RB;
        const int nr = I.R - r0 < BC_RB ? I.R - r0 : BC_RB;
        const int sigma = I.far_rows[loc % nrows];
        const int q2 = I.q2, cw = I.helm ? 2 : 1;
        const int G = blockDim.x / q2;
        const int t = threadIdx.x, gg = t / q2, a = t % q2;
        float sr[BC_RB], si[BC_RB];
#pragma unroll
        for (int j = 0; j < BC_RB; ++j) sr[j] = si[j] = 0.0f;
        if (gg < G) {
            const float4 X = reinterpret_cast<const float4*>(I.igeo32)[(int64_t)sigma * q2 + a];
            const int64_t rstride = (int64_t)I.C * q2 * cw;      // between right-hand sides
            const float* xr = I.xh + (int64_t)r0 * rstride;
            for (int64_t blk = I.far_ptr[sigma] + gg; blk < I.far_ptr[sigma + 1]; blk += G) {
                const int64_t tau = I.far_src[blk];
                const float4* Y = reinterpret_cast<const float4*>(I.igeo32) + tau * q2;
                const float* V = xr + tau * q2 * cw;
                for (int b = 0; b < q2; ++b) {
                    const float4 y = Y[b];
                    const float d0 = X.x - y.x, d1 = X.y - y.y, d2 = X.z - y.z;
                    const float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
                    const float rinv = rsqrtf(r2);
                    const float w = y.w * rinv;
                    if (cw == 2) {
                        // phase reduced to [-pi, pi] first: the hardware sine and
                        // cosine are accurate on that interval only
                        float ph = I.kappa * (r2 * rinv);
                        ph = fmaf(-6.283185307179586f, rintf(ph * 0.15915494309189535f), ph);
                        float sn, cs;
                        __sincosf(ph, &sn, &cs);
                        const float kr = w * cs, ki = w * sn;
#pragma unroll
                        for (int j = 0; j < BC_RB; ++j) {
                            if (j < nr) {
                                const float vr = V[j * rstride + 2 * b], vi = V[j * rstride + 2 * b + 1];
                                sr[j] = fmaf(kr, vr, fmaf(-ki, vi, sr[j]));
                                si[j] = fmaf(kr, vi, fmaf(ki, vr, si[j]));
                            }
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < BC_RB; ++j)
                            if (j < nr) sr[j] = fmaf(w, V[j * rstride + b], sr[j]);
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < BC_RB; ++j) {
            red[2 * (j * blockDim.x + t)] = sr[j];
            red[2 * (j * blockDim.x + t) + 1] = si[j];
        }
        __syncthreads();
        if (t < q2) {
            const float ka = reinterpret_cast<const float4*>(I.igeo32)[(int64_t)sigma * q2 + t].w * 0.07957747154594767f;
            for (int j = 0; j < nr; ++j) {
                float vr = 0.0f, vi = 0.0f;
                for (int g = 0; g < G; ++g) {
                    vr += red[2 * (j * blockDim.x + g * q2 + t)];
                    vi += red[2 * (j * blockDim.x + g * q2 + t) + 1];
                }
                float* o = I.yh + (((int64_t)(r0 + j) * I.C + sigma) * q2 + t) * cw;
                o[0] = vr * ka;
                if (cw == 2) o[1] = vi * ka;
            }
        }
        __syncthreads();
    }
}

// L2L for children at level kk of every instance with m >= kk; item (r, cl, b)
__global__ void b_l2l_kernel(const BatchInst* __restrict__ B, int n, const int64_t* __restrict__ pre, int64_t total,
                             int kk) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int k = find_inst(pre, n, g);
    const BatchInst& I = B[k];
    const int64_t nL1 = I.lvl[kk + 1] - I.lvl[kk];
    int64_t loc = g - pre[k];
    const int b = (int)(loc % I.q2);
    loc /= I.q2;
    const int64_t cl = loc % nL1;
    const int r = (int)(loc / nL1);
    const int q = I.q, q2 = I.q2, bu = b % q, bv = b / q, c = (int)(cl & 3), cw = I.helm ? 2 : 1;
    const float* Su = I.Sf + (c & 1) * q2;
    const float* Sv = I.Sf + (c >> 1) * q2;
    const float* v = I.yh + (((int64_t)r * I.C + I.lvl[kk - 1] + cl / 4) * q2) * cw;
    float ar = 0.0f, ai = 0.0f;
    for (int av = 0; av < q; ++av) {
        float tr = 0.0f, ti = 0.0f;
        for (int au = 0; au < q; ++au) {
            tr = fmaf(Su[au * q + bu], v[(av * q + au) * cw], tr);
            if (cw == 2) ti = fmaf(Su[au * q + bu], v[(av * q + au) * 2 + 1], ti);
        }
        ar = fmaf(Sv[av * q + bv], tr, ar);
        ai = fmaf(Sv[av * q + bv], ti, ai);
    }
    float* o = I.yh + (((int64_t)r * I.C + I.lvl[kk] + cl) * q2 + b) * cw;
    o[0] += ar;
    if (cw == 2) o[1] += ai;
}

// back-projection plus near field; item (r, e, i)
__global__ void b_back_near_kernel(const BatchInst* __restrict__ B, int n, const int64_t* __restrict__ pre,
                                   int64_t total) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int k = find_inst(pre, n, g);
    const BatchInst& I = B[k];
    int64_t loc = g - pre[k];
    const int i = (int)(loc % I.nb);
    loc /= I.nb;
    const int64_t e = loc % I.E;
    const int r = (int)(loc / I.E);
    const int iu = i % I.pp, iv = i / I.pp, cw = I.helm ? 2 : 1, nbb = I.nb * I.nb;
    float ar = 0.0f, ai = 0.0f;
    const float* v = I.yh + (((int64_t)r * I.C + I.lvl[I.m] + e) * I.q2) * cw;
    for (int av = 0; av < I.q; ++av)
        for (int au = 0; au < I.q; ++au) {
            const float c = I.Mf[au * I.pp + iu] * I.Mf[av * I.pp + iv];
            ar = fmaf(c, v[(av * I.q + au) * cw], ar);
            if (cw == 2) ai = fmaf(c, v[(av * I.q + au) * 2 + 1], ai);
        }
    const float* xr = I.xs + (int64_t)r * I.E * I.nb * cw;
    for (int64_t kb = I.near_ptr[e]; kb < I.near_ptr[e + 1]; ++kb) {
        const float* xv = xr + (int64_t)I.near_src[kb] * I.nb * cw;
        for (int j = 0; j < I.nb; ++j) {
            if (cw == 2) {
                const float br = I.near32[2 * (kb * nbb + i * I.nb + j)], bi = I.near32[2 * (kb * nbb + i * I.nb + j) + 1];
                ar = fmaf(br, xv[2 * j], fmaf(-bi, xv[2 * j + 1], ar));
                ai = fmaf(br, xv[2 * j + 1], fmaf(bi, xv[2 * j], ai));
            } else {
                ar = fmaf(I.near32[kb * nbb + i * I.nb + j], xv[j], ar);
            }
        }
    }
    float* o = I.ys + (((int64_t)r * I.E + e) * I.nb + i) * cw;
    o[0] = ar;
    if (cw == 2) o[1] = ai;
}

// y = T y*; item (r, dof)
__global__ void b_restrict_kernel(const BatchInst* __restrict__ B, int n, const int64_t* __restrict__ pre,
                                  int64_t total, double* __restrict__ y) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int k = find_inst(pre, n, g);
    const BatchInst& I = B[k];
    int64_t loc = g - pre[k];
    const int64_t dof = loc % I.N;
    const int r = (int)(loc / I.N);
    const int patch = (int)(dof / ((int64_t)I.n1 * I.n1));
    const int rem = (int)(dof % ((int64_t)I.n1 * I.n1));
    const int jv = rem / I.n1, ju = rem % I.n1, p = I.p, pp = I.pp, cw = I.helm ? 2 : 1;
    const int64_t per = (int64_t)I.ne1 * I.ne1;
    float ar = 0.0f, ai = 0.0f;
    for (int iy = jv - p; iy <= jv; ++iy) {
        if (iy < 0 || iy >= I.ne1) continue;
        for (int ix = ju - p; ix <= ju; ++ix) {
            if (ix < 0 || ix >= I.ne1) continue;
            const int64_t e = patch * per + morton2(ix, iy);
            const float* v = I.ys + ((int64_t)r * I.E + e) * I.nb * cw;
            for (int iv = 0; iv < pp; ++iv)
                for (int iu = 0; iu < pp; ++iu) {
                    const float c = (float)I.ext[((int64_t)ix * pp + (ju - ix)) * pp + iu] *
                                    (float)I.ext[((int64_t)iy * pp + (jv - iy)) * pp + iv];
                    ar = fmaf(c, v[(iv * pp + iu) * cw], ar);
                    if (cw == 2) ai = fmaf(c, v[(iv * pp + iu) * 2 + 1], ai);
                }
        }
    }
    double* o = y + I.xoff + ((int64_t)r * I.N + dof) * cw;
    o[0] = ar;
    if (cw == 2) o[1] = ai;
}

namespace {

// all stages of one application, on b->stream (also used for graph capture)
cudaError_t batch_enqueue(ibem_batch* b, const double* x, double* y, int coupling_threads) {
    using B = ibem_batch;
    cudaStream_t st = b->stream;
    const int T = 256;
    int launches = 0;
    auto total = [&](int s) { return b->pre[s][b->n]; };
    cudaError_t e;
    if ((e = cudaMemsetAsync(b->arena + b->yh_begin, 0, b->yh_floats * sizeof(float), st))) return e;
    if ((e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), st))) return e;
    if (total(B::ST_LIFT) > 0) {
        b_lift_kernel<<<bblk(total(B::ST_LIFT), T), T, 0, st>>>(b->d_inst, b->n, b->d_pre[B::ST_LIFT], total(B::ST_LIFT), x);
        ++launches;
    }
    if (total(B::ST_LEAF) > 0) {
        b_leaf_kernel<<<bblk(total(B::ST_LEAF), T), T, 0, st>>>(b->d_inst, b->n, b->d_pre[B::ST_LEAF], total(B::ST_LEAF));
        ++launches;
    }
    for (int kk = 1; kk <= b->max_m; ++kk) {
        const int s = B::ST_FIXED + 2 * (kk - 1);
        if (total(s) == 0) continue;
        b_m2m_kernel<<<bblk(total(s), T), T, 0, st>>>(b->d_inst, b->n, b->d_pre[s], total(s), kk);
        ++launches;
    }
    if (total(B::ST_COUPLE) > 0) {
        const size_t sm = 2 * (size_t)b->couple_rb * coupling_threads * sizeof(float);
        if (b->couple_rb == 4)
            b_coupling_kernel<4><<<b->couple_ctas, coupling_threads, sm, st>>>(
                b->d_inst, b->n, b->d_pre[B::ST_COUPLE], total(B::ST_COUPLE), b->d_counter);
        else if (b->couple_rb == 16)
            b_coupling_kernel<16><<<b->couple_ctas, coupling_threads, sm, st>>>(
                b->d_inst, b->n, b->d_pre[B::ST_COUPLE], total(B::ST_COUPLE), b->d_counter);
        else
            b_coupling_kernel<8><<<b->couple_ctas, coupling_threads, sm, st>>>(
                b->d_inst, b->n, b->d_pre[B::ST_COUPLE], total(B::ST_COUPLE), b->d_counter);
        ++launches;
    }
    for (int kk = 1; kk <= b->max_m; ++kk) {
        const int s = B::ST_FIXED + 2 * (kk - 1) + 1;
        if (total(s) == 0) continue;
        b_l2l_kernel<<<bblk(total(s), T), T, 0, st>>>(b->d_inst, b->n, b->d_pre[s], total(s), kk);
        ++launches;
    }
    if (total(B::ST_BACK) > 0) {
        b_back_near_kernel<<<bblk(total(B::ST_BACK), T), T, 0, st>>>(b->d_inst, b->n, b->d_pre[B::ST_BACK],
                                                                     total(B::ST_BACK));
        ++launches;
    }
    if (total(B::ST_RESTRICT) > 0) {
        b_restrict_kernel<<<bblk(total(B::ST_RESTRICT), T), T, 0, st>>>(b->d_inst, b->n, b->d_pre[B::ST_RESTRICT],
                                                                        total(B::ST_RESTRICT), y);
        ++launches;
    }
    b->launches = launches;
    return cudaGetLastError();
}

}  // namespace
}  // namespace ibem

using namespace ibem;

extern "C" {

ibem_status ibem_batch_create(ibem_handle* const* handles, int n, const int* nrhs, void* cuda_stream,
                              ibem_batch** out) {
    if (!out || !handles || !nrhs || n <= 0) return IBEM_ERR_ARG;
    *out = nullptr;
    ibem_batch* b = new ibem_batch();
    b->n = n;
    b->stream = (cudaStream_t)cuda_stream;
    if (!b->stream) {
        // graph capture needs a stream other than the legacy default stream
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return IBEM_ERR_CUDA;
        }
        b->own_stream = true;
    }
    b->handles.assign(handles, handles + n);
    cudaGetDevice(&b->device);
    b->offsets.assign(n + 1, 0);
    size_t floats = 0;
    std::vector<size_t> base(n);
    for (int i = 0; i < n; ++i) {
        ibem_handle* h = handles[i];
        if (!h || !h->assembled || h->device != b->device || h->P.q == 0 || nrhs[i] < 1 || nrhs[i] > 256 ||
            h->P.q > 8) {
            if (b->own_stream) cudaStreamDestroy(b->stream);
            delete b;
            return IBEM_ERR_ARG;
        }
        const Plan& P = h->P;
        const int cw = h->helm ? 2 : 1;
        b->offsets[i + 1] = b->offsets[i] + (int64_t)nrhs[i] * P.N * cw;
        base[i] = floats;
        floats += (size_t)nrhs[i] * cw * (2 * P.Nstar);       // xs, ys
        b->max_m = std::max(b->max_m, P.m);
    }
    b->yh_begin = floats;
    for (int i = 0; i < n; ++i) {
        const Plan& P = handles[i]->P;
        floats += (size_t)nrhs[i] * (handles[i]->helm ? 2 : 1) * P.C * P.q2;   // yh (cleared per application)
    }
    b->yh_floats = floats - b->yh_begin;
    std::vector<size_t> xh_base(n);
    for (int i = 0; i < n; ++i) {
        const Plan& P = handles[i]->P;
        xh_base[i] = floats;
        floats += (size_t)nrhs[i] * (handles[i]->helm ? 2 : 1) * P.C * P.q2;
    }
    b->arena_floats = floats;
    if (cudaMalloc(&b->arena, floats * sizeof(float)) || cudaMalloc(&b->d_counter, sizeof(int))) {
        ibem_batch_destroy(b);
        return IBEM_ERR_OOM;
    }
    size_t yh_cursor = b->yh_begin;
    for (int i = 0; i < n; ++i) {
        ibem_handle* h = handles[i];
        const Plan& P = h->P;
        const int cw = h->helm ? 2 : 1;
        BatchInst I;
        std::memset(&I, 0, sizeof(I));
        I.helm = h->helm ? 1 : 0;
        I.p = P.p; I.pp = P.pp; I.nb = P.nb; I.ne1 = P.ne1; I.n1 = P.n1; I.q = P.q; I.q2 = P.q2; I.m = P.m;
        I.R = nrhs[i];
        I.kappa = (float)P.prm.kappa;
        I.E = P.E; I.N = P.N; I.Nstar = P.Nstar; I.C = P.C;
        for (size_t l = 0; l < P.level_off.size() && l < 12; ++l) I.lvl[l] = P.level_off[l];
        I.ext = h->d_ext; I.Mf = h->d_Mf; I.Sf = h->d_Sf;
        I.near_ptr = h->d_near_ptr; I.near_src = h->d_near_src; I.near32 = h->d_near32;
        I.far_ptr = h->d_far_ptr; I.far_src = h->d_far_src; I.far_rows = h->d_far_rows;
        I.igeo32 = h->d_igeo32;
        I.xs = b->arena + base[i];
        I.ys = I.xs + (size_t)I.R * cw * P.Nstar;
        I.yh = b->arena + yh_cursor;
        yh_cursor += (size_t)I.R * cw * P.C * P.q2;
        I.xh = b->arena + xh_base[i];
        I.xoff = b->offsets[i];
        b->inst.push_back(I);
    }
    // stage work lists
    const int nst = ibem_batch::ST_FIXED + 2 * b->max_m;
    b->pre.assign(nst, std::vector<int64_t>(n + 1, 0));
    for (int i = 0; i < n; ++i) {
        const BatchInst& I = b->inst[i];
        const int64_t R = I.R;
        int64_t cnt[64] = {0};
        cnt[ibem_batch::ST_LIFT] = R * I.E * I.nb;
        cnt[ibem_batch::ST_LEAF] = R * I.E * I.q2;
        cnt[ibem_batch::ST_BACK] = R * I.E * I.nb;
        cnt[ibem_batch::ST_NEAR] = 0;
        cnt[ibem_batch::ST_RESTRICT] = R * I.N;
        cnt[ibem_batch::ST_COUPLE] = ((R + 7) / 8) * (int64_t)handles[i]->far_rows.size();   // RB = 8 until tuned
        for (int kk = 1; kk <= b->max_m; ++kk) {
            if (I.m >= kk) {
                const int L = I.m - kk;
                cnt[ibem_batch::ST_FIXED + 2 * (kk - 1)] = R * (I.lvl[L + 1] - I.lvl[L]) * I.q2;
                cnt[ibem_batch::ST_FIXED + 2 * (kk - 1) + 1] = R * (I.lvl[kk + 1] - I.lvl[kk]) * I.q2;
            }
        }
        for (int s = 0; s < nst; ++s) b->pre[s][i + 1] = b->pre[s][i] + cnt[s];
    }
    b->d_pre.assign(nst, nullptr);
    bool fail = cudaMalloc(&b->d_inst, n * sizeof(BatchInst)) != cudaSuccess;
    if (!fail) cudaMemcpyAsync(b->d_inst, b->inst.data(), n * sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream);
    for (int s = 0; s < nst && !fail; ++s) {
        fail = cudaMalloc(&b->d_pre[s], (n + 1) * sizeof(int64_t)) != cudaSuccess;
        if (!fail)
            cudaMemcpyAsync(b->d_pre[s], b->pre[s].data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, b->stream);
    }
    if (fail) {
        ibem_batch_destroy(b);
        return IBEM_ERR_OOM;
    }
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    // coupling work list (items of RB right-hand sides) for every candidate tile
    auto couple_list = [&](int rb) {
        std::vector<int64_t> pre(n + 1, 0);
        for (int i = 0; i < n; ++i)
            pre[i + 1] = pre[i] + (int64_t)((b->inst[i].R + rb - 1) / rb) * (int64_t)handles[i]->far_rows.size();
        return pre;
    };
    auto use_tile = [&](int rb) {
        b->couple_rb = rb;
        b->pre[ibem_batch::ST_COUPLE] = couple_list(rb);
        cudaMemcpyAsync(b->d_pre[ibem_batch::ST_COUPLE], b->pre[ibem_batch::ST_COUPLE].data(), (n + 1) * sizeof(int64_t),
                        cudaMemcpyHostToDevice, b->stream);
    };
    auto resident = [&](int rb, int threads) {
        const size_t smb = 2 * (size_t)rb * threads * sizeof(float);
        int per_sm = 0;
        if (rb == 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b_coupling_kernel<4>, threads, smb);
        else if (rb == 16) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b_coupling_kernel<16>, threads, smb);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b_coupling_kernel<8>, threads, smb);
        return sms * per_sm;   // 0: this shape cannot be launched (registers or shared memory)
    };
    cudaFuncSetAttribute(b_coupling_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4 * 512 * 4);
    cudaFuncSetAttribute(b_coupling_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 8 * 512 * 4);
    cudaFuncSetAttribute(b_coupling_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 16 * 512 * 4);
    // autotune the tile (right-hand sides per work item) and the CTA size of the
    // persistent coupling kernel on scratch inputs
    double* xs_tmp = nullptr;
    double* ys_tmp = nullptr;
    const int64_t tot = b->offsets[n];
    int best_rb = 8;
    if (cudaMallocAsync(&xs_tmp, tot * sizeof(double), b->stream) == cudaSuccess &&
        cudaMallocAsync(&ys_tmp, tot * sizeof(double), b->stream) == cudaSuccess) {
        cudaMemsetAsync(xs_tmp, 0, tot * sizeof(double), b->stream);
        float best = 1e30f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int rb : {4, 8, 16}) {
            use_tile(rb);
            for (int threads : {128, 256, 512}) {
                b->couple_ctas = resident(rb, threads);
                if (b->couple_ctas == 0) continue;
                // a shape whose launch fails takes no time: never a candidate
                if (batch_enqueue(b, xs_tmp, ys_tmp, threads) != cudaSuccess) continue;
                cudaEventRecord(e0, b->stream);
                if (batch_enqueue(b, xs_tmp, ys_tmp, threads) != cudaSuccess) continue;
                cudaEventRecord(e1, b->stream);
                cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                b->tune_ms.push_back(ms);
                if (ms < best) {
                    best = ms;
                    b->couple_threads = threads;
                    best_rb = rb;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFreeAsync(xs_tmp, b->stream);
        cudaFreeAsync(ys_tmp, b->stream);
    }
    use_tile(best_rb);
    b->couple_ctas = resident(best_rb, b->couple_threads);
    if (b->couple_ctas == 0) {
        ibem_batch_destroy(b);
        return IBEM_ERR_CUDA;
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        ibem_batch_destroy(b);
        return IBEM_ERR_CUDA;
    }
    *out = b;
    return IBEM_OK;
}

ibem_status ibem_batch_offsets(const ibem_batch* b, int64_t* offsets) {
    if (!b || !offsets) return IBEM_ERR_ARG;
    for (int i = 0; i <= b->n; ++i) offsets[i] = b->offsets[i];
    return IBEM_OK;
}

ibem_status ibem_batch_matvec(ibem_batch* b, const double* x_dev, double* y_dev) {
    if (!b || !x_dev || !y_dev || x_dev == y_dev) return IBEM_ERR_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return IBEM_ERR_CUDA;
    if (!b->exec || b->graph_x != x_dev || b->graph_y != y_dev) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return IBEM_ERR_CUDA;
        cudaError_t e = batch_enqueue(b, x_dev, y_dev, b->couple_threads);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &b->graph);
        if (e != cudaSuccess || e2 != cudaSuccess) return IBEM_ERR_CUDA;
        if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) return IBEM_ERR_CUDA;
        b->graph_x = x_dev;
        b->graph_y = y_dev;
    }
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return IBEM_ERR_CUDA;
    return IBEM_OK;
}

ibem_status ibem_batch_info(const ibem_batch* b, int* launches_per_apply, int* coupling_threads,
                            int* coupling_rhs_tile) {
    if (!b) return IBEM_ERR_ARG;
    if (launches_per_apply) *launches_per_apply = b->launches;
    if (coupling_threads) *coupling_threads = b->couple_threads;
    if (coupling_rhs_tile) *coupling_rhs_tile = b->couple_rb;
    return IBEM_OK;
}

ibem_status ibem_batch_destroy(ibem_batch* b) {
    if (!b) return IBEM_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->arena);
    cudaFree(b->d_counter);
    cudaFree(b->solve_x);
    cudaFree(b->solve_y);
    cudaFree(b->d_inst);
    for (auto p : b->d_pre) cudaFree(p);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return IBEM_OK;
}

}  // extern "C"
