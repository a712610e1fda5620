// Operator application of libibem: y = T [A_near + U K V^T] T^T x (Sec. 4.2,
// Sec. 4.3), plus right-hand side and potential evaluation.
//
// Steps of one application (each a kernel below):
//   lift       x* = T^T x            Bezier extraction per element
//   moments    x^_e = (M (x) M) x*_e  leaf moments int L_a B_i (geometry-free)
//   M2M        x^_P = sum_c (S_c (x) S_c) x^_c   level by level, leaves to root
//   coupling   y^_s = sum_t K_st x^_t             every far block, all levels
//   L2L        y^_c += (S_c (x) S_c)^T y^_P       root to leaves
//   back       y*_e = (M (x) M)^T y^_e
//   near       y*_e += sum_{e'} B_{e e'} x*_{e'}  stored near-field blocks
//   restrict   y = T y*
// S_c[a][b] = L_a((c + z_b) / 2) re-expands a parent Lagrange polynomial in the
// child's basis exactly (degree q-1), so nested and non-nested moments agree.
#include "ibem_internal.cuh"

namespace ibem {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ inline void elem_coords(int64_t e, int ne1, int* patch, int* ix, int* iy) {
    int64_t per = (int64_t)ne1 * ne1;
    *patch = (int)(e / per);
    uint32_t x, y;
    morton2_inv((uint32_t)(e % per), &x, &y);
    *ix = (int)x;
    *iy = (int)y;
}

// ---- T^T and T ---------------------------------------------------------------
__global__ void lift_kernel(int R, int64_t E, int p, int ne1, const double* __restrict__ ext,
                            const double* __restrict__ x, int64_t N, double* __restrict__ xs) {
    int pp = p + 1, nb = pp * pp, n1 = ne1 + p;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R * E * nb) return;
    int64_t r = idx / (E * nb);
    int64_t rem = idx % (E * nb);
    int64_t e = rem / nb;
    int i = (int)(rem % nb), iu = i % pp, iv = i / pp;
    int patch, ix, iy;
    elem_coords(e, ne1, &patch, &ix, &iy);
    const double* xp = x + r * N + (int64_t)patch * n1 * n1;
    double acc = 0.0;
    for (int r2 = 0; r2 < pp; ++r2) {
        double cv = ext[((int64_t)iy * pp + r2) * pp + iv];
        double row = 0.0;
        for (int r1 = 0; r1 < pp; ++r1) row += ext[((int64_t)ix * pp + r1) * pp + iu] * xp[(iy + r2) * n1 + ix + r1];
        acc += cv * row;
    }
    xs[idx] = acc;
}

__global__ void restrict_kernel(int R, int64_t N, int p, int ne1, const double* __restrict__ ext,
                                const double* __restrict__ ys, int64_t E, double* __restrict__ y) {
    int pp = p + 1, nb = pp * pp, n1 = ne1 + p;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R * N) return;
    int64_t r = idx / N, dof = idx % N;
    int patch = (int)(dof / ((int64_t)n1 * n1));
    int rem = (int)(dof % ((int64_t)n1 * n1));
    int jv = rem / n1, ju = rem % n1;
    int64_t per = (int64_t)ne1 * ne1;
    double acc = 0.0;
    for (int iy = jv - p; iy <= jv; ++iy) {
        if (iy < 0 || iy >= ne1) continue;
        for (int ix = ju - p; ix <= ju; ++ix) {
            if (ix < 0 || ix >= ne1) continue;
            const double* v = ys + (r * E + patch * per + morton2(ix, iy)) * nb;
            const double* cu = ext + ((int64_t)ix * pp + (ju - ix)) * pp;
            const double* cv = ext + ((int64_t)iy * pp + (jv - iy)) * pp;
            for (int iv = 0; iv < pp; ++iv) {
                double row = 0.0;
                for (int iu = 0; iu < pp; ++iu) row += cu[iu] * v[iv * pp + iu];
                acc += cv[iv] * row;
            }
        }
    }
    y[idx] = acc;
}

// ---- upward pass -------------------------------------------------------------
__global__ void leaf_moment_kernel(int R, int64_t E, int pp, int q, const double* __restrict__ M,
                                   const double* __restrict__ xs, int64_t leaf_off, int64_t C,
                                   double* __restrict__ xh) {
    int q2 = q * q, nb = pp * pp;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R * E * q2) return;
    int64_t r = idx / (E * q2);
    int64_t rem = idx % (E * q2);
    int64_t e = rem / q2;
    int a = (int)(rem % q2), au = a % q, av = a / q;
    const double* v = xs + (r * E + e) * nb;
    double acc = 0.0;
    for (int iv = 0; iv < pp; ++iv) {
        double row = 0.0;
        for (int iu = 0; iu < pp; ++iu) row += M[au * pp + iu] * v[iv * pp + iu];
        acc += M[av * pp + iv] * row;
    }
    xh[(r * C + leaf_off + e) * q2 + a] = acc;
}

__global__ void m2m_kernel(int R, int64_t nL, int64_t offL, int64_t offL1, int q, const double* __restrict__ S,
                           int64_t C, double* __restrict__ xh) {
    int q2 = q * q;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R * nL * q2) return;
    int64_t r = idx / (nL * q2);
    int64_t rem = idx % (nL * q2);
    int64_t pl = rem / q2;
    int a = (int)(rem % q2), au = a % q, av = a / q;
    double acc = 0.0;
    for (int c = 0; c < 4; ++c) {
        const double* Su = S + (c & 1) * q2;
        const double* Sv = S + (c >> 1) * q2;
        const double* v = xh + (r * C + offL1 + 4 * pl + c) * q2;
        for (int bv = 0; bv < q; ++bv) {
            double row = 0.0;
            for (int bu = 0; bu < q; ++bu) row += Su[au * q + bu] * v[bv * q + bu];
            acc += Sv[av * q + bv] * row;
        }
    }
    xh[(r * C + offL + pl) * q2 + a] = acc;
}

// Separable M2M: one CTA per parent; T_c[bv][au] = sum_bu S_cx[au][bu] x_c[bv][bu],
// x^_P[av][au] = sum_c sum_bv S_cy[av][bv] T_c[bv][au].
__global__ void m2m_sep_kernel(int64_t nL, int64_t offL, int64_t offL1, int q, const double* __restrict__ S,
                               int64_t C, double* __restrict__ xh) {
    __shared__ double xc[4 * IBEM_MAX_Q * IBEM_MAX_Q], Tc[4 * IBEM_MAX_Q * IBEM_MAX_Q];
    const int q2 = q * q;
    const int64_t pl = blockIdx.x, r = blockIdx.y;
    const double* src = xh + (r * C + offL1 + 4 * pl) * q2;
    for (int i = threadIdx.x; i < 4 * q2; i += blockDim.x) xc[i] = src[i];
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * q2; i += blockDim.x) {
        int c = i / q2, rem = i % q2, bv = rem / q, au = rem % q;
        const double* Su = S + (c & 1) * q2 + au * q;
        const double* v = xc + c * q2 + bv * q;
        double acc = 0.0;
        for (int bu = 0; bu < q; ++bu) acc += Su[bu] * v[bu];
        Tc[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < q2; i += blockDim.x) {
        int av = i / q, au = i % q;
        double acc = 0.0;
        for (int c = 0; c < 4; ++c) {
            const double* Sv = S + (c >> 1) * q2 + av * q;
            for (int bv = 0; bv < q; ++bv) acc += Sv[bv] * Tc[c * q2 + bv * q + au];
        }
        xh[(r * C + offL + pl) * q2 + i] = acc;
    }
}

// Separable L2L: one CTA per parent; U_cx[av][bu] = sum_au S_cx[au][bu] y_P[av][au],
// y_c[bv][bu] += sum_av S_cy[av][bv] U_cx[av][bu] for the 4 children.
__global__ void l2l_sep_kernel(int64_t nL, int64_t offL, int64_t offL1, int q, const double* __restrict__ S,
                               int64_t C, double* __restrict__ yh) {
    __shared__ double yp[IBEM_MAX_Q * IBEM_MAX_Q], U[2 * IBEM_MAX_Q * IBEM_MAX_Q];
    const int q2 = q * q;
    const int64_t pl = blockIdx.x, r = blockIdx.y;
    for (int i = threadIdx.x; i < q2; i += blockDim.x) yp[i] = yh[(r * C + offL + pl) * q2 + i];
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * q2; i += blockDim.x) {
        int cx = i / q2, rem = i % q2, av = rem / q, bu = rem % q;
        const double* Su = S + cx * q2;
        double acc = 0.0;
        for (int au = 0; au < q; ++au) acc += Su[au * q + bu] * yp[av * q + au];
        U[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * q2; i += blockDim.x) {
        int c = i / q2, rem = i % q2, bv = rem / q, bu = rem % q;
        const double* Sv = S + (c >> 1) * q2;
        const double* u = U + (c & 1) * q2;
        double acc = 0.0;
        for (int av = 0; av < q; ++av) acc += Sv[av * q + bv] * u[av * q + bu];
        yh[(r * C + offL1 + 4 * pl + c) * q2 + rem] += acc;
    }
}

// ---- coupling, FP64, stored K ------------------------------------------------
// One CTA per target cluster with far blocks; thread t = 4 a + s accumulates
// row a over columns b = s + 4 kk of every block, then the 4 lanes of a row
// are summed with shuffles.  K is laid out so that each kk step is one
// contiguous 4 q2-double read across the CTA.
__global__ void coupling64_kernel(const int32_t* __restrict__ rows, const int64_t* __restrict__ fptr,
                                  const int32_t* __restrict__ fsrc, const double* __restrict__ K, int q2, int kpt,
                                  int64_t C, const double* __restrict__ xh, double* __restrict__ yh) {
    int sigma = rows[blockIdx.x];
    int64_t r = blockIdx.y;
    int t = threadIdx.x, s = t & 3, a = t >> 2;
    bool active = t < 4 * q2;
    double acc = 0.0;
    if (active) {
        int64_t b0 = fptr[sigma], b1 = fptr[sigma + 1];
        const double* xr = xh + r * C * q2;
        for (int64_t blk = b0; blk < b1; ++blk) {
            const double* Kb = K + blk * (int64_t)kpt * 4 * q2 + t;
            const double* xt = xr + (int64_t)fsrc[blk] * q2;
            for (int kk = 0; kk < kpt; ++kk) {
                int b = s + 4 * kk;
                if (b < q2) acc += Kb[(int64_t)kk * 4 * q2] * xt[b];
            }
        }
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (active && s == 0) yh[(r * C + sigma) * q2 + a] = acc;
}

// ---- coupling, FP64-accurate in double-float arithmetic on the FP32 pipe -------
// Same thread layout and K layout as coupling64_kernel.  K = kh + kl and
// x^ = xh + xl are float pairs; kh*xh is formed exactly (p + e, e from an FMA),
// the cross terms kh*xl + kl*xh are added to e, and (p, e) is accumulated with
// Knuth's TwoSum.  Each block's double-float partial sum is folded into an FP64
// accumulator, so FP64 work is a few operations per block instead of one FMA
// per matrix entry.
// x^ (rows of q2 doubles) -> (hi, lo) float pairs in rows of q2p >= q2 (q2p even,
// so every row starts on a 16-byte boundary for the bulk copies).
__global__ void split_kernel(int64_t rows, int q2, int q2p, const double* __restrict__ x, float2* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * q2p) return;
    int64_t row = i / q2p;
    int c = (int)(i % q2p);
    double v = c < q2 ? x[row * q2 + c] : 0.0;
    float hi = (float)v;
    out[i] = make_float2(hi, (float)(v - (double)hi));
}

// The CTA of target cluster sigma streams the coupling matrices of its row -
// contiguous in HBM - through a ring of NST shared-memory stages with 1-D bulk
// copies (cp.async.bulk, one elected thread) completed on mbarriers; all
// threads compute from shared memory, so the copies of the next NST blocks are
// in flight while one block is consumed.  Every wait is bounded by
// `wait_limit` polls; on a timeout the CTA records IBEM_DEVICE_TIMEOUT in
// *status, waits (bounded) for its copies in flight and returns.
__device__ inline unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ inline void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ inline void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ inline bool mbar_wait(uint64_t* bar, unsigned parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Laplace coupling matrices are symmetric, K_{tau sigma} = K_{sigma tau}^T (the
// kernel and the product of surface measures are symmetric and evaluated
// identically), so only the blocks with sigma < tau are stored.  The CTA of
// row sigma streams them once and uses each twice: rows give
// y^_sigma = sum K x^_tau (register accumulation, stored at the end), columns
// give the block's share K^T x^_sigma of y^_tau (reduced across the 4 lanes
// that share a column and stored per block in `colpart`); column_gather_kernel
// then adds the shares to every y^_tau in a fixed order, so the result is
// deterministic.  Both passes read K from the shared-memory stage.
__device__ inline void df_add(float& hi, float& lo, float h2, float l2) {
    float s = hi + h2;
    float z = s - hi;
    float err = (hi - (s - z)) + (h2 - z);
    hi = s;
    lo = lo + l2 + err;
}

__device__ inline void df_fma(float kh, float kl, float xh, float xl, float& hi, float& lo) {
    float p = kh * xh;
    float e = fmaf(kh, xh, -p);
    e = fmaf(kh, xl, e);
    e = fmaf(kl, xh, e);
    df_add(hi, lo, p, e);
}

// EXACT: q2 == 4 KPT (even q), so every lane's columns and rows exist and the
// strides are compile-time constants.
template <int KPT, int NST, bool EXACT>
__global__ void coupling_df_kernel(const int32_t* __restrict__ rows, const int64_t* __restrict__ fptr,
                                   const int32_t* __restrict__ fsrc, const float2* __restrict__ K, int q2_rt,
                                   int q2p, int maxrow, int64_t C, const float2* __restrict__ xh,
                                   double* __restrict__ yh, float2* __restrict__ colpart, int64_t nblk_total,
                                   long long wait_limit, int* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem[];
    // [0, 128): mbarriers; then the row's source clusters; then NST stages of
    // (coupling block, source moments)
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    int32_t* srcs = reinterpret_cast<int32_t*>(smem + 128);
    const int q2 = EXACT ? 4 * KPT : q2_rt;
    const int stride = 4 * q2;
    const int belems = KPT * stride;
    const int selems = belems + q2p;
    float2* stage = reinterpret_cast<float2*>(smem + 128 + (((size_t)maxrow * 4 + 15) / 16) * 16);
    const unsigned kbytes = (unsigned)belems * 8u, xbytes = (unsigned)q2p * 8u;
    const int sigma = rows[blockIdx.x];
    const int64_t r = blockIdx.y;
    const int t = threadIdx.x, s = t & 3, a = t >> 2;   // row pass: row a, columns s + 4 kk
    const int bc = t >> 2, sc = t & 3;                   // column pass: column bc, rows sc + 4 j
    const bool active = t < stride;
    const int64_t b0 = fptr[sigma];
    const int n = (int)(fptr[sigma + 1] - b0);
    const float2* xr = xh + r * C * q2p;
    for (int j = t; j < n; j += blockDim.x) srcs[j] = fsrc[b0 + j];
    float2 xs[KPT];
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        int row = sc + 4 * j;
        xs[j] = (active && (EXACT || row < q2)) ? xr[(int64_t)sigma * q2p + row] : make_float2(0.f, 0.f);
    }
    if (t == 0) {
        for (int i = 0; i < NST; ++i) mbar_init(&full[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (t == 0) {
        for (int i = 0; i < NST && i < n; ++i) {
            float2* dst = stage + (size_t)i * selems;
            mbar_expect_tx(&full[i], kbytes + xbytes);
            bulk_load(dst, K + (b0 + i) * (int64_t)belems, kbytes, &full[i]);
            bulk_load(dst + belems, xr + (int64_t)srcs[i] * q2p, xbytes, &full[i]);
        }
    }
    // FP64 work is kept off the per-block path (GB300's FP64 unit is narrow):
    // the row sum stays double-float and is folded into `acc` every 8 blocks.
    double acc = 0.0;
    float rh = 0.0f, rl = 0.0f;
    int i = 0;
    bool failed = false;
    for (; i < n; ++i) {
        const int st = i % NST;
        const bool ok = mbar_wait(&full[st], (unsigned)((i / NST) & 1), wait_limit);
        float ch = 0.0f, cl = 0.0f;
        if (ok && active) {
            const float2* Kb = stage + (size_t)st * selems;
            const float2* xt = Kb + belems;
            float hi = 0.0f, lo = 0.0f;
#pragma unroll
            for (int kk = 0; kk < KPT; ++kk) {
                int b = s + 4 * kk;
                if (EXACT || b < q2) {
                    float2 kv = Kb[kk * stride + t];
                    float2 x = xt[b];
                    df_fma(kv.x, kv.y, x.x, x.y, hi, lo);
                }
            }
            df_add(rh, rl, hi, lo);
            if ((i & 7) == 7) {
                acc += (double)rh + (double)rl;
                rh = 0.0f;
                rl = 0.0f;
            }
            const float2* Kc = Kb + (bc >> 2) * stride + (bc & 3) + 4 * sc;
#pragma unroll
            for (int j = 0; j < KPT; ++j) {
                if (EXACT || sc + 4 * j < q2) {
                    float2 kv = Kc[16 * j];
                    df_fma(kv.x, kv.y, xs[j].x, xs[j].y, ch, cl);
                }
            }
        }
        // columns: combine the 4 lanes that share column bc (all lanes take part)
#pragma unroll
        for (int off = 1; off <= 2; off <<= 1) {
            float oh = __shfl_xor_sync(0xffffffffu, ch, off);
            float ol = __shfl_xor_sync(0xffffffffu, cl, off);
            df_add(ch, cl, oh, ol);
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (t == 0 && i + NST < n) {
            float2* dst = stage + (size_t)st * selems;
            mbar_expect_tx(&full[st], kbytes + xbytes);
            bulk_load(dst, K + (b0 + i + NST) * (int64_t)belems, kbytes, &full[st]);
            bulk_load(dst + belems, xr + (int64_t)srcs[i + NST] * q2p, xbytes, &full[st]);
        }
        if (active && sc == 0) colpart[(r * nblk_total + b0 + i) * q2 + bc] = make_float2(ch, cl);
    }
    acc += (double)rh + (double)rl;
    if (failed) {
        if (t == 0) {
            atomicOr(status, 1);
            // drain: every issued copy must land before the CTA's shared memory is released
            for (int j = i; j < n && j < i + NST; ++j) mbar_wait(&full[j % NST], (unsigned)((j / NST) & 1), 1LL << 24);
        }
        __syncthreads();
        return;
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (active && s == 0) yh[(r * C + sigma) * q2 + a] = acc;
}

// y^_tau += sum over the stored blocks (sigma, tau), sigma < tau, of their column
// shares, in the order of the transposed list.
__global__ void column_gather_kernel(int R, int64_t C, int q2, const int64_t* __restrict__ tptr,
                                     const int32_t* __restrict__ tblk, const float2* __restrict__ colpart,
                                     int64_t nblk_total, double* __restrict__ yh) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)R * C * q2) return;
    int64_t r = idx / (C * q2);
    int64_t rem = idx % (C * q2);
    int64_t tau = rem / q2;
    int b = (int)(rem % q2);
    if (tptr[tau + 1] == tptr[tau]) return;
    float hi = 0.0f, lo = 0.0f;
#pragma unroll 4
    for (int64_t k = tptr[tau]; k < tptr[tau + 1]; ++k) {
        float2 v = colpart[(r * nblk_total + tblk[k]) * q2 + b];
        df_add(hi, lo, v.x, v.y);
    }
    yh[(r * C + tau) * q2 + b] += (double)hi + (double)lo;
}

// ---- coupling, FP32, kernel generated on the fly ------------------------------
// src32[t][b] = (x, y, z, k_b x^_b / (4 pi)) of every cluster; one CTA per target
// cluster; thread (g, a) handles target point a against blocks g, g + NS, ...;
// the per-block float sums are accumulated in double.
__global__ void src32_kernel(int64_t n, const float* __restrict__ igeo32, const double* __restrict__ xh,
                             float4* __restrict__ src) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* g = igeo32 + 4 * i;
    src[i] = make_float4(g[0], g[1], g[2], (float)((double)g[3] * xh[i] * (1.0 / (4.0 * IBEM_PI))));
}

// Thread (g, ap) evaluates target rows ap and ap + half against the blocks
// g, g + G, ... of the row, so every source point loaded serves two rows; the
// per-block float sums are accumulated in double and the G partial sums are
// combined through shared memory.
__global__ void coupling32_kernel(const int32_t* __restrict__ rows, const int64_t* __restrict__ fptr,
                                  const int32_t* __restrict__ fsrc, const float* __restrict__ igeo32,
                                  const float4* __restrict__ src, int q2, int G, double* __restrict__ yh) {
    extern __shared__ double red[];
    const int sigma = rows[blockIdx.x];
    const int t = threadIdx.x;
    const int half = (q2 + 1) >> 1;
    const int g = t / half, ap = t % half;
    const int a0 = ap, a1 = ap + half;
    const bool two = a1 < q2;
    double acc0 = 0.0, acc1 = 0.0;
    if (g < G) {
        const float* X0 = igeo32 + 4 * ((int64_t)sigma * q2 + a0);
        const float* X1 = igeo32 + 4 * ((int64_t)sigma * q2 + (two ? a1 : a0));
        const float x0 = X0[0], y0 = X0[1], z0 = X0[2];
        const float x1 = X1[0], y1 = X1[1], z1 = X1[2];
        const int64_t b0 = fptr[sigma], b1 = fptr[sigma + 1];
        for (int64_t blk = b0 + g; blk < b1; blk += G) {
            const float4* Y = src + (int64_t)fsrc[blk] * q2;
            float f0 = 0.0f, f1 = 0.0f, h0 = 0.0f, h1 = 0.0f;
            int b = 0;
            for (; b + 1 < q2; b += 2) {
                float4 u = Y[b], v = Y[b + 1];
                float d0 = x0 - u.x, d1 = y0 - u.y, d2 = z0 - u.z;
                float e0 = x1 - u.x, e1 = y1 - u.y, e2 = z1 - u.z;
                float c0 = x0 - v.x, c1 = y0 - v.y, c2 = z0 - v.z;
                float k0 = x1 - v.x, k1 = y1 - v.y, k2 = z1 - v.z;
                f0 = fmaf(u.w, rsqrtf(d0 * d0 + d1 * d1 + d2 * d2), f0);
                f1 = fmaf(u.w, rsqrtf(e0 * e0 + e1 * e1 + e2 * e2), f1);
                h0 = fmaf(v.w, rsqrtf(c0 * c0 + c1 * c1 + c2 * c2), h0);
                h1 = fmaf(v.w, rsqrtf(k0 * k0 + k1 * k1 + k2 * k2), h1);
            }
            if (b < q2) {
                float4 u = Y[b];
                float d0 = x0 - u.x, d1 = y0 - u.y, d2 = z0 - u.z;
                float e0 = x1 - u.x, e1 = y1 - u.y, e2 = z1 - u.z;
                f0 = fmaf(u.w, rsqrtf(d0 * d0 + d1 * d1 + d2 * d2), f0);
                f1 = fmaf(u.w, rsqrtf(e0 * e0 + e1 * e1 + e2 * e2), f1);
            }
            acc0 += (double)(f0 + h0);
            acc1 += (double)(f1 + h1);
        }
    }
    if (g < G) {
        red[g * q2 + a0] = acc0;
        if (two) red[g * q2 + a1] = acc1;
    }
    __syncthreads();
    if (t < q2) {
        double v = 0.0;
        for (int k = 0; k < G; ++k) v += red[k * q2 + t];
        yh[(int64_t)sigma * q2 + t] = v * (double)igeo32[4 * ((int64_t)sigma * q2 + t) + 3];
    }
}

// ---- downward pass -----------------------------------------------------------
__global__ void l2l_kernel(int R, int64_t nL1, int64_t offL, int64_t offL1, int q, const double* __restrict__ S,
                           int64_t C, double* __restrict__ yh) {
    int q2 = q * q;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R * nL1 * q2) return;
    int64_t r = idx / (nL1 * q2);
    int64_t rem = idx % (nL1 * q2);
    int64_t cl = rem / q2;
    int b = (int)(rem % q2), bu = b % q, bv = b / q;
    int c = (int)(cl & 3);
    const double* Su = S + (c & 1) * q2;
    const double* Sv = S + (c >> 1) * q2;
    const double* v = yh + (r * C + offL + cl / 4) * q2;
    double acc = 0.0;
    for (int av = 0; av < q; ++av) {
        double row = 0.0;
        for (int au = 0; au < q; ++au) row += Su[au * q + bu] * v[av * q + au];
        acc += Sv[av * q + bv] * row;
    }
    yh[(r * C + offL1 + cl) * q2 + b] += acc;
}

__global__ void leaf_back_kernel(int R, int64_t E, int pp, int q, const double* __restrict__ M,
                                 const double* __restrict__ yh, int64_t leaf_off, int64_t C,
                                 double* __restrict__ ys) {
    int q2 = q * q, nb = pp * pp;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R * E * nb) return;
    int64_t r = idx / (E * nb);
    int64_t rem = idx % (E * nb);
    int64_t e = rem / nb;
    int i = (int)(rem % nb), iu = i % pp, iv = i / pp;
    const double* v = yh + (r * C + leaf_off + e) * q2;
    double acc = 0.0;
    for (int av = 0; av < q; ++av) {
        double row = 0.0;
        for (int au = 0; au < q; ++au) row += M[au * pp + iu] * v[av * q + au];
        acc += M[av * pp + iv] * row;
    }
    ys[idx] = acc;
}

// ---- near field product ------------------------------------------------------
// One CTA per target element; thread t = i * nb + j accumulates B[i][j] x*_s[j]
// over the row's blocks (one coalesced nb^2 read per block), then rows are
// summed through shared memory.  The row's source elements are staged in shared
// memory (so a source value's load does not wait for a dependent global load)
// and the sum over blocks runs in four independent partial sums.
template <typename T>
__global__ void near_apply_kernel(const int64_t* __restrict__ nptr, const int32_t* __restrict__ nsrc,
                                  const T* __restrict__ blocks, int nb, int64_t E, const T* __restrict__ xs,
                                  double* __restrict__ ys) {
    extern __shared__ double red[];
    __shared__ int32_t srcs[256];
    const int64_t e = blockIdx.x, r = blockIdx.y;
    const int t = threadIdx.x, nbb = nb * nb;
    const int64_t k0 = nptr[e], k1 = nptr[e + 1];
    const int j = t % nb;
    const T* xr = xs + r * E * nb;
    T p0 = (T)0, p1 = (T)0, p2 = (T)0, p3 = (T)0;
    for (int64_t kb = k0; kb < k1; kb += 256) {
        const int kc = (int)(k1 - kb < 256 ? k1 - kb : 256);
        __syncthreads();   // the previous chunk's source list is consumed
        for (int i = t; i < kc; i += blockDim.x) srcs[i] = nsrc[kb + i];
        __syncthreads();
        if (t < nbb) {
            const T* bk = blocks + kb * nbb + t;
            int kk = 0;
            for (; kk + 3 < kc; kk += 4) {
                p0 += bk[(int64_t)kk * nbb] * xr[(int64_t)srcs[kk] * nb + j];
                p1 += bk[(int64_t)(kk + 1) * nbb] * xr[(int64_t)srcs[kk + 1] * nb + j];
                p2 += bk[(int64_t)(kk + 2) * nbb] * xr[(int64_t)srcs[kk + 2] * nb + j];
                p3 += bk[(int64_t)(kk + 3) * nbb] * xr[(int64_t)srcs[kk + 3] * nb + j];
            }
            for (; kk < kc; ++kk) p0 += bk[(int64_t)kk * nbb] * xr[(int64_t)srcs[kk] * nb + j];
        }
    }
    red[t] = t < nbb ? (double)((p0 + p1) + (p2 + p3)) : 0.0;
    __syncthreads();
    if (t < nb) {
        double v = 0.0;
        for (int jj = 0; jj < nb; ++jj) v += red[t * nb + jj];
        ys[(r * E + e) * nb + t] += v;
    }
}

__global__ void d2f_kernel(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

cudaError_t ensure_workspace(ibem_handle* h, int nrhs) {
    // nrhs counts real right-hand sides (a complex one counts twice)
    if (nrhs <= h->ws_nrhs) return cudaSuccess;
    Plan& P = h->P;
    if (h->helm) {
        cudaFree(h->d_hsx); cudaFree(h->d_hsy); cudaFree(h->d_xh4);
        h->d_hsx = h->d_hsy = nullptr;
        h->d_xh4 = nullptr;
    }
    cudaFree(h->d_xs); cudaFree(h->d_ys); cudaFree(h->d_xh); cudaFree(h->d_yh);
    cudaFree(h->d_xs32); cudaFree(h->d_src32); cudaFree(h->d_xh2);
    h->d_xh2 = nullptr;
    h->d_xs = h->d_ys = h->d_xh = h->d_yh = nullptr;
    h->d_xs32 = nullptr;
    h->d_src32 = nullptr;
    h->ws_nrhs = 0;
    cudaError_t e;
    size_t ns = (size_t)nrhs * P.Nstar, nh = (size_t)nrhs * P.C * (P.q2 > 0 ? P.q2 : 1);
    if ((e = cudaMalloc(&h->d_xs, ns * sizeof(double)))) return e;
    if ((e = cudaMalloc(&h->d_ys, ns * sizeof(double)))) return e;
    if ((e = cudaMalloc(&h->d_xh, nh * sizeof(double)))) return e;
    if ((e = cudaMalloc(&h->d_yh, nh * sizeof(double)))) return e;
    if ((e = cudaMalloc(&h->d_xh2, (size_t)nrhs * P.C * ((P.q2 + 1) & ~1) * sizeof(float2) + 16))) return e;
    cudaFree(h->d_colpart);
    h->d_colpart = nullptr;
    // column shares of the stored symmetric Laplace coupling only (a Helmholtz
    // handle never reads them; at 64 right-hand sides they would need n_up q^2
    // 128 floats pairs)
    if (!h->helm && h->d_Kdf &&
        (e = cudaMalloc(&h->d_colpart, (size_t)nrhs * (h->n_up > 0 ? h->n_up : 1) * (P.q2 > 0 ? P.q2 : 1) *
                                           sizeof(float2))))
        return e;
    if ((e = cudaMalloc(&h->d_xs32, ns * sizeof(float)))) return e;
    if ((e = cudaMalloc(&h->d_src32, (size_t)P.C * (P.q2 > 0 ? P.q2 : 1) * sizeof(float4)))) return e;
    if (h->helm) {
        size_t n = (size_t)(P.N > P.nq ? P.N : P.nq);
        if ((e = cudaMalloc(&h->d_hsx, (size_t)nrhs * n * sizeof(double)))) return e;
        if ((e = cudaMalloc(&h->d_hsy, (size_t)nrhs * P.N * sizeof(double)))) return e;
        // double-float moments of the stored coupling only (none when it is generated)
        if (h->d_Kc && (e = cudaMalloc(&h->d_xh4, (size_t)(nrhs / 2 + 1) * P.C * ((P.q2 + 1) & ~1) * sizeof(float4) + 32)))
            return e;
    }
    h->ws_nrhs = nrhs;
    return cudaSuccess;
}



namespace {

template <int KPT, int NST, bool EXACT>
cudaError_t launch_df_t(ibem_handle* h, int R) {
    const int q2 = h->P.q2, q2p = (q2 + 1) & ~1;
    const int threads = ((4 * q2 + 31) / 32) * 32;
    const size_t sbytes = ((size_t)KPT * 4 * q2 + q2p) * sizeof(float2);
    const size_t head = 128 + (((size_t)h->max_up_row * 4 + 15) / 16) * 16;
    const size_t sm = head + (size_t)NST * sbytes;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(coupling_df_kernel<KPT, NST, EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm)))
        return e;
    dim3 grid((unsigned)h->up_rows.size(), R);
    coupling_df_kernel<KPT, NST, EXACT><<<grid, threads, sm, h->stream>>>(
        h->d_up_rows, h->d_up_ptr, h->d_up_src, h->d_Kdf, q2, q2p, h->max_up_row, h->P.C, h->d_xh2, h->d_yh,
        h->d_colpart, h->n_up, h->wait_limit, h->d_status);
    return cudaGetLastError();
}

// Ring depths instantiated per KPT for even q (q = 2, 4, 6, 8, 10, 12).
std::vector<int> df_depth_candidates(int kpt) {
    switch (kpt) {
        case 1: return {4, 8};
        case 4: return {4, 6};
        case 9: return {2, 3, 4};
        case 16: return {2, 3};
        case 25: return {2};
        case 36: return {1};
        default: return {};
    }
}

}  // namespace

cudaError_t launch_coupling_df(ibem_handle* h, int R, int nst) {
    if (4 * h->kpt == h->P.q2) {
        if (nst == 0) nst = df_depth_candidates(h->kpt).back();
        switch (h->kpt * 16 + nst) {
            case 1 * 16 + 4: return launch_df_t<1, 4, true>(h, R);
            case 1 * 16 + 8: return launch_df_t<1, 8, true>(h, R);
            case 4 * 16 + 4: return launch_df_t<4, 4, true>(h, R);
            case 4 * 16 + 6: return launch_df_t<4, 6, true>(h, R);
            case 9 * 16 + 2: return launch_df_t<9, 2, true>(h, R);
            case 9 * 16 + 3: return launch_df_t<9, 3, true>(h, R);
            case 9 * 16 + 4: return launch_df_t<9, 4, true>(h, R);
            case 16 * 16 + 2: return launch_df_t<16, 2, true>(h, R);
            case 16 * 16 + 3: return launch_df_t<16, 3, true>(h, R);
            case 25 * 16 + 2: return launch_df_t<25, 2, true>(h, R);
            case 36 * 16 + 1: return launch_df_t<36, 1, true>(h, R);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (h->kpt) {
        case 3: return launch_df_t<3, 8, false>(h, R);
        case 7: return launch_df_t<7, 4, false>(h, R);
        case 13: return launch_df_t<13, 3, false>(h, R);
        case 21: return launch_df_t<21, 2, false>(h, R);
        case 31: return launch_df_t<31, 1, false>(h, R);
        default: return cudaErrorInvalidValue;
    }
}

// Autotuner of the ring depth (even q): every candidate depth whose shared
// memory fits is run twice on the handle's own stored matrices (moments set to
// zero) and the fastest second run is kept.  Called once, at the end of
// assembly, outside any stream capture.
cudaError_t tune_coupling_df(ibem_handle* h) {
    h->df_nst = 0;
    if (4 * h->kpt != h->P.q2) return cudaSuccess;
    const int q2 = h->P.q2, q2p = (q2 + 1) & ~1;
    const size_t sbytes = ((size_t)h->kpt * 4 * q2 + q2p) * sizeof(float2);
    const size_t head = 128 + (((size_t)h->max_up_row * 4 + 15) / 16) * 16;
    std::vector<int> depths;
    for (int n : df_depth_candidates(h->kpt))
        if (head + (size_t)n * sbytes <= 227 * 1024) depths.push_back(n);
    if (depths.empty()) return cudaErrorInvalidValue;
    h->df_nst = depths.back();
    if (depths.size() == 1) return cudaSuccess;
    cudaError_t e;
    if ((e = ensure_workspace(h, 1))) return e;
    if ((e = cudaMemsetAsync(h->d_xh2, 0, (size_t)h->P.C * q2p * sizeof(float2), h->stream))) return e;
    cudaEvent_t a, b;
    if ((e = cudaEventCreate(&a))) return e;
    if ((e = cudaEventCreate(&b))) {
        cudaEventDestroy(a);
        return e;
    }
    float best = 1e30f;
    for (int n : depths) {
        if ((e = launch_coupling_df(h, 1, n))) break;
        cudaEventRecord(a, h->stream);
        if ((e = launch_coupling_df(h, 1, n))) break;
        cudaEventRecord(b, h->stream);
        if ((e = cudaEventSynchronize(b))) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best) {
            best = ms;
            h->df_nst = n;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e;
}

cudaError_t apply_operator(ibem_handle* h, const double* x, double* y, int nrhs, int precision) {
    Plan& P = h->P;
    cudaStream_t st = h->stream;
    cudaError_t e;
    if (precision == IBEM_FP32 && mr_supported(h, nrhs)) return apply_operator_mrhs(h, x, y, nrhs);
    // the FP64 Laplace coupling needs stored matrices (absent with IBEM_COUPLING_NONE)
    if (!h->helm && precision == IBEM_FP64 && P.q > 0 && !h->far_rows.empty() && !h->d_K && !h->d_Kdf)
        return cudaErrorInvalidValue;
    if (h->helm) {
        if ((e = ensure_workspace(h, 2 * nrhs))) return e;
        h->applications++;
        return helm_apply_operator(h, x, y, nrhs, precision, h->d_hsx, h->d_hsy);
    }
    if ((e = ensure_workspace(h, nrhs))) return e;
    const int R = nrhs;
    const int T = 256;
    h->applications++;
    {
        PhaseTimer pt(h, 0);
        lift_kernel<<<nblk(R * P.E * P.nb, T), T, 0, st>>>(R, P.E, P.p, P.ne1, h->d_ext, x, P.N, h->d_xs);
        h->launches++;
    }
    if (P.q > 0) {
        const int q2 = P.q2;
        const int64_t leaf_off = P.level_off[P.m];
        {
            PhaseTimer pt(h, 1);
            leaf_moment_kernel<<<nblk(R * P.E * q2, T), T, 0, st>>>(R, P.E, P.pp, P.q, h->d_M, h->d_xs, leaf_off,
                                                                     P.C, h->d_xh);
            h->launches++;
            for (int L = P.m - 1; L >= 0; --L) {
                int64_t nL = P.level_off[L + 1] - P.level_off[L];
                m2m_sep_kernel<<<dim3((unsigned)nL, R), 64, 0, st>>>(nL, P.level_off[L], P.level_off[L + 1], P.q,
                                                                    h->d_S, P.C, h->d_xh);
                h->launches++;
            }
            if ((e = cudaMemsetAsync(h->d_yh, 0, (size_t)R * P.C * q2 * sizeof(double), st))) return e;
        }
        unsigned nrows = (unsigned)h->far_rows.size();
        if (nrows > 0) {
            PhaseTimer pt(h, 2);
            if (precision == IBEM_FP32) {
                const int half = (q2 + 1) / 2;
                int ns = 256 / half > 0 ? 256 / half : 1;
                int threads = ((ns * half + 31) / 32) * 32;
                for (int r = 0; r < R; ++r) {
                    src32_kernel<<<nblk(P.C * q2, T), T, 0, st>>>(P.C * q2, h->d_igeo32, h->d_xh + (size_t)r * P.C * q2,
                                                                  h->d_src32);
                    coupling32_kernel<<<nrows, threads, (size_t)ns * q2 * sizeof(double), st>>>(
                        h->d_far_rows, h->d_far_ptr, h->d_far_src, h->d_igeo32, h->d_src32, q2, ns,
                        h->d_yh + (size_t)r * P.C * q2);
                    h->launches += 2;
                }
            } else if (h->d_K) {
                int threads = ((4 * q2 + 31) / 32) * 32;
                coupling64_kernel<<<dim3(nrows, R), threads, 0, st>>>(h->d_far_rows, h->d_far_ptr, h->d_far_src, h->d_K,
                                                                      q2, h->kpt, P.C, h->d_xh, h->d_yh);
                h->launches++;
            } else {
                const int q2p = (q2 + 1) & ~1;
                split_kernel<<<nblk(R * P.C * q2p, T), T, 0, st>>>(R * P.C, q2, q2p, h->d_xh, h->d_xh2);
                if ((e = launch_coupling_df(h, R, h->df_nst))) return e;
                column_gather_kernel<<<nblk((int64_t)R * P.C * q2, T), T, 0, st>>>(R, P.C, q2, h->d_tr_ptr, h->d_tr_blk,
                                                                                   h->d_colpart, h->n_up, h->d_yh);
                h->launches++;
                h->launches += 2;
            }
        }
        PhaseTimer pt(h, 3);
        for (int L = 0; L < P.m; ++L) {
            int64_t nL = P.level_off[L + 1] - P.level_off[L];
            l2l_sep_kernel<<<dim3((unsigned)nL, R), 64, 0, st>>>(nL, P.level_off[L], P.level_off[L + 1], P.q, h->d_S,
                                                                P.C, h->d_yh);
            h->launches++;
        }
        leaf_back_kernel<<<nblk(R * P.E * P.nb, T), T, 0, st>>>(R, P.E, P.pp, P.q, h->d_M, h->d_yh, leaf_off, P.C,
                                                                 h->d_ys);
        h->launches++;
    } else {
        if ((e = cudaMemsetAsync(h->d_ys, 0, (size_t)R * P.Nstar * sizeof(double), st))) return e;
    }
    int threads = ((P.nb * P.nb + 31) / 32) * 32;
    {
        PhaseTimer pt(h, 4);
        if (precision == IBEM_FP32) {
            d2f_kernel<<<nblk(R * P.Nstar, T), T, 0, st>>>(h->d_xs, h->d_xs32, R * P.Nstar);
            near_apply_kernel<float><<<dim3((unsigned)P.E, R), threads, threads * sizeof(double), st>>>(
                h->d_near_ptr, h->d_near_src, h->d_near32, P.nb, P.E, h->d_xs32, h->d_ys);
            h->launches += 2;
        } else {
            near_apply_kernel<double><<<dim3((unsigned)P.E, R), threads, threads * sizeof(double), st>>>(
                h->d_near_ptr, h->d_near_src, h->d_near, P.nb, P.E, h->d_xs, h->d_ys);
            h->launches++;
        }
    }
    {
        PhaseTimer pt(h, 5);
        restrict_kernel<<<nblk(R * P.N, 32), 32, 0, st>>>(R, P.N, P.p, P.ne1, h->d_ext, h->d_ys, P.E, y);
        h->launches++;
    }
    return cudaGetLastError();
}

// ---- right-hand side -----------------------------------------------------------
// g*_e[i] = sum_g W_g Phi[g][i] g(x_g), then b = T g*.
__global__ void rhs_super_kernel(int R, int64_t E, int QQ, int nb, const double* __restrict__ qgeo,
                                 const double* __restrict__ phi, const double* __restrict__ g, int64_t nq,
                                 double* __restrict__ gs) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R * E * nb) return;
    int64_t r = idx / (E * nb);
    int64_t rem = idx % (E * nb);
    int64_t e = rem / nb;
    int i = (int)(rem % nb);
    double acc = 0.0;
    for (int q = 0; q < QQ; ++q) acc += qgeo[4 * (e * QQ + q) + 3] * phi[q * nb + i] * g[r * nq + e * QQ + q];
    gs[idx] = acc;
}

cudaError_t launch_rhs(ibem_handle* h, const double* g, int nrhs, double* b) {
    Plan& P = h->P;
    cudaError_t e;
    if (h->helm) {
        if ((e = ensure_workspace(h, 2 * nrhs))) return e;
        return helm_launch_rhs(h, g, nrhs, b, h->d_hsx, h->d_hsy);
    }
    if ((e = ensure_workspace(h, nrhs))) return e;
    const int T = 256;
    int QQ = P.Q * P.Q;
    rhs_super_kernel<<<nblk(nrhs * P.E * P.nb, T), T, 0, h->stream>>>(nrhs, P.E, QQ, P.nb, h->d_qgeo, h->d_phi, g,
                                                                       P.nq, h->d_ys);
    restrict_kernel<<<nblk(nrhs * P.N, T), T, 0, h->stream>>>(nrhs, P.N, P.p, P.ne1, h->d_ext, h->d_ys, P.E, b);
    return cudaGetLastError();
}

// ---- potential -------------------------------------------------------------------
// u(x) = sum_e sum_g W_g w_h(x_g) / (4 pi |x - x_g|).  The densities at the Gauss
// points are formed first; then every thread owns one evaluation point and a
// slice of the sources, and slices are combined with atomics.
__global__ void density_kernel(int64_t E, int QQ, int nb, const double* __restrict__ qgeo,
                               const double* __restrict__ phi, const double* __restrict__ ws,
                               double4_32a* __restrict__ srcs) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= E * QQ) return;
    int64_t e = idx / QQ;
    int q = (int)(idx % QQ);
    double mu = 0.0;
    for (int i = 0; i < nb; ++i) mu += phi[q * nb + i] * ws[e * nb + i];
    const double* X = qgeo + 4 * idx;
    srcs[idx] = make_double4_32a(X[0], X[1], X[2], X[3] * mu / (4.0 * IBEM_PI));
}

__global__ void potential_kernel(int64_t npts, const double* __restrict__ pts, int64_t nsrc,
                                 const double4_32a* __restrict__ srcs, int64_t chunk, double* __restrict__ u) {
    int64_t ip = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= npts) return;
    double x0 = pts[3 * ip], x1 = pts[3 * ip + 1], x2 = pts[3 * ip + 2];
    int64_t s0 = blockIdx.y * chunk, s1 = s0 + chunk < nsrc ? s0 + chunk : nsrc;
    double acc = 0.0;
    for (int64_t s = s0; s < s1; ++s) {
        double4_32a y = srcs[s];
        double d0 = x0 - y.x, d1 = x1 - y.y, d2 = x2 - y.z;
        acc += y.w / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
    atomicAdd(u + ip, acc);
}

// Direct Laplace potential on caller-provided work space: ws holds the lifted
// density of one right-hand side (ndof_super doubles), srcs the Gauss-point
// sources (E Q^2); u is cleared and accumulated with atomics over chunks of
// sources.  Shared by ibem_potential and the allocation-free entry point.
cudaError_t launch_potential_ws(ibem_handle* h, const double* w, int nrhs, const double* pts, int64_t npts,
                                double* u, double* ws, double4_32a* srcs) {
    Plan& P = h->P;
    cudaError_t e;
    if ((e = cudaMemsetAsync(u, 0, (size_t)nrhs * npts * sizeof(double), h->stream))) return e;
    if (npts <= 0) return cudaSuccess;
    const int T = 256;
    const int QQ = P.Q * P.Q;
    const int64_t nsrc = P.E * QQ;
    int64_t nsplit = (608 * 128) / npts;
    if (nsplit < 1) nsplit = 1;
    if (nsplit > 65535) nsplit = 65535;
    const int64_t chunk = (nsrc + nsplit - 1) / nsplit;
    nsplit = (nsrc + chunk - 1) / chunk;
    for (int r = 0; r < nrhs; ++r) {
        lift_kernel<<<nblk(P.E * P.nb, T), T, 0, h->stream>>>(1, P.E, P.p, P.ne1, h->d_ext, w + (size_t)r * P.N, P.N,
                                                              ws);
        density_kernel<<<nblk(nsrc, T), T, 0, h->stream>>>(P.E, QQ, P.nb, h->d_qgeo, h->d_phi, ws, srcs);
        potential_kernel<<<dim3(nblk(npts, 128), (unsigned)nsplit), 128, 0, h->stream>>>(npts, pts, nsrc, srcs, chunk,
                                                                                         u + (size_t)r * npts);
        if ((e = cudaGetLastError())) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_potential(ibem_handle* h, const double* w, int nrhs, const double* pts, int64_t npts,
                             double* u) {
    Plan& P = h->P;
    cudaError_t e;
    if (h->helm) {
        if ((e = ensure_workspace(h, 2 * nrhs))) return e;
        return helm_launch_potential(h, w, nrhs, pts, npts, u, h->d_hsx);
    }
    if ((e = ensure_workspace(h, 1))) return e;
    double4_32a* srcs = nullptr;
    if ((e = cudaMallocAsync(&srcs, (size_t)P.E * P.Q * P.Q * sizeof(double4_32a), h->stream))) return e;
    e = launch_potential_ws(h, w, nrhs, pts, npts, u, h->d_xs, srcs);
    cudaFreeAsync(srcs, h->stream);
    return e;
}

}  // namespace ibem
