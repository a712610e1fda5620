// Many right-hand sides at once (FP32 operator): y = T A T^T x for R right-hand
// sides with the far-field coupling contracted on the 5th-generation tensor
// cores (Sec. 4.2: with R columns the coupling y^_s += K_st x^_t is a dense
// GEMM).
//
// Layouts put the right-hand side innermost: x* [E][nb][R], x^ [C][q2][R],
// y* [E][nb][R]; values are float (Laplace) or float2 (Helmholtz).
//
// Coupling on tcgen05: one CTA per target cluster sigma.  For every far block
// the CTA evaluates K_{sigma tau} in FP32 (rsqrt, phase reduced to [-pi, pi],
// sine and cosine) and writes it as BF16 into a shared-memory A tile, in the
// real form [[Kr, -Ki], [Ki, Kr]] for Helmholtz, padded to MAP = 128 rows and
// KAP (multiple of 16) columns.  The B tile - the moments x^_tau as BF16 in the
// same form, RP (multiple of 16) right-hand sides - is prepared once per
// application in global memory and fetched with one cp.async.bulk per block.
// Both tiles are double-buffered; one thread issues tcgen05.mma (kind::f16,
// BF16 inputs, FP32 accumulation) into a TMEM accumulator [MAP lanes][RP
// columns] that persists over the whole far row, and tcgen05.commit signals an
// mbarrier when a buffer may be reused.  Tiles use the no-swizzle K-major
// layout: 8 x 8 core matrices of 128 contiguous bytes, LBO = 128 bytes along
// K, SBO = (KAP / 8) * 128 bytes along M or N.  All waits are bounded.
#include <cuda_bf16.h>

#include <algorithm>

#include "ibem_internal.cuh"

namespace ibem {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <bool CPLX> struct MrType { typedef float T; };
template <> struct MrType<true> { typedef float2 T; };

__device__ inline float mr_zero(float) { return 0.0f; }
__device__ inline float2 mr_zero(float2) { return make_float2(0.0f, 0.0f); }
__device__ inline float mr_axpy(float a, float x, float y) { return fmaf(a, x, y); }
__device__ inline float2 mr_axpy(float a, float2 x, float2 y) { return make_float2(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y)); }

// ---- layout conversion ---------------------------------------------------------------
// x [R][N] doubles (interleaved complex) -> xt [N][R]
template <bool CPLX>
__global__ void mr_in_kernel(int R, int64_t N, const double* __restrict__ x, typename MrType<CPLX>::T* __restrict__ xt) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)R * N) return;
    int64_t n = idx / R;
    int r = (int)(idx % R);
    if constexpr (CPLX) xt[idx] = make_float2((float)x[2 * (r * N + n)], (float)x[2 * (r * N + n) + 1]);
    else xt[idx] = (float)x[r * N + n];
}

// ---- T^T, moments, M2M ----------------------------------------------------------------
template <bool CPLX>
__global__ void mr_lift_kernel(int R, int64_t E, int p, int ne1, const double* __restrict__ ext,
                               const typename MrType<CPLX>::T* __restrict__ xt, typename MrType<CPLX>::T* __restrict__ xs) {
    typedef typename MrType<CPLX>::T T;
    const int pp = p + 1, nb = pp * pp, n1 = ne1 + p;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= E * nb * R) return;
    int r = (int)(idx % R);
    int64_t rem = idx / R;
    int i = (int)(rem % nb);
    int64_t e = rem / nb;
    int64_t per = (int64_t)ne1 * ne1;
    int patch = (int)(e / per);
    uint32_t ix, iy;
    morton2_inv((uint32_t)(e % per), &ix, &iy);
    const int iu = i % pp, iv = i / pp;
    T acc = mr_zero(T());
    for (int r2 = 0; r2 < pp; ++r2) {
        float cv = (float)ext[((int64_t)iy * pp + r2) * pp + iv];
        for (int r1 = 0; r1 < pp; ++r1) {
            float c = cv * (float)ext[((int64_t)ix * pp + r1) * pp + iu];
            int64_t dof = (int64_t)patch * n1 * n1 + (int64_t)(iy + r2) * n1 + (ix + r1);
            acc = mr_axpy(c, xt[dof * R + r], acc);
        }
    }
    xs[idx] = acc;
}

template <bool CPLX>
__global__ void mr_leaf_kernel(int R, int64_t E, int pp, int q, const float* __restrict__ M,
                               const typename MrType<CPLX>::T* __restrict__ xs, int64_t leaf_off,
                               typename MrType<CPLX>::T* __restrict__ xh) {
    typedef typename MrType<CPLX>::T T;
    const int q2 = q * q, nb = pp * pp;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= E * q2 * R) return;
    int r = (int)(idx % R);
    int64_t rem = idx / R;
    int a = (int)(rem % q2);
    int64_t e = rem / q2;
    const int au = a % q, av = a / q;
    T acc = mr_zero(T());
    for (int iv = 0; iv < pp; ++iv)
        for (int iu = 0; iu < pp; ++iu)
            acc = mr_axpy(M[au * pp + iu] * M[av * pp + iv], xs[(e * nb + iv * pp + iu) * R + r], acc);
    xh[((leaf_off + e) * q2 + a) * R + r] = acc;
}

// Separable M2M, one CTA per (parent, chunk of RC right-hand sides):
// T_c[bv][au] = sum_bu S_cx[au][bu] x_c[bv][bu], x_P[av][au] = sum_c sum_bv S_cy[av][bv] T_c[bv][au].
constexpr int MR_RC = 8;
template <bool CPLX>
__global__ void mr_m2m_sep_kernel(int R, int64_t offL, int64_t offL1, int q, const float* __restrict__ S,
                                  typename MrType<CPLX>::T* __restrict__ xh) {
    typedef typename MrType<CPLX>::T T;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int q2 = q * q;
    T* xc = reinterpret_cast<T*>(sm_raw);               // [4][q2][RC]
    T* Tc = xc + 4 * q2 * MR_RC;                        // [4][q][q][RC]
    float* Ss = reinterpret_cast<float*>(Tc + 4 * q2 * MR_RC);   // [2][q][q]
    const int64_t pl = blockIdx.x;
    const int r0 = blockIdx.y * MR_RC;
    const int rc = R - r0 < MR_RC ? R - r0 : MR_RC;
    for (int i = threadIdx.x; i < 2 * q2; i += blockDim.x) Ss[i] = S[i];
    for (int i = threadIdx.x; i < 4 * q2 * MR_RC; i += blockDim.x) {
        const int r = i % MR_RC, cb = i / MR_RC;        // cb = c * q2 + b
        xc[i] = r < rc ? xh[((offL1 + 4 * pl) * q2 + cb) * R + r0 + r] : mr_zero(T());
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * q2 * MR_RC; i += blockDim.x) {
        const int r = i % MR_RC, rest = i / MR_RC;
        const int c = rest / q2, bv = (rest % q2) / q, au = rest % q;
        const float* Su = Ss + (c & 1) * q2 + au * q;
        const T* v = xc + (c * q2 + bv * q) * MR_RC + r;
        T acc = mr_zero(T());
        for (int bu = 0; bu < q; ++bu) acc = mr_axpy(Su[bu], v[bu * MR_RC], acc);
        Tc[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < q2 * MR_RC; i += blockDim.x) {
        const int r = i % MR_RC, a = i / MR_RC, av = a / q, au = a % q;
        if (r >= rc) continue;
        T acc = mr_zero(T());
        for (int c = 0; c < 4; ++c) {
            const float* Sv = Ss + (c >> 1) * q2 + av * q;
            const T* tv = Tc + (c * q2 + au) * MR_RC + r;
            for (int bv = 0; bv < q; ++bv) acc = mr_axpy(Sv[bv], tv[bv * q * MR_RC], acc);
        }
        xh[((offL + pl) * q2 + a) * R + r0 + r] = acc;
    }
}

// Separable L2L, one CTA per (parent, chunk): U_cx[av][bu] = sum_au S_cx[au][bu] y_P[av][au],
// y_c[bv][bu] += sum_av S_cy[av][bv] U_cx[av][bu].
template <bool CPLX>
__global__ void mr_l2l_sep_kernel(int R, int64_t offL, int64_t offL1, int q, const float* __restrict__ S,
                                  typename MrType<CPLX>::T* __restrict__ yh) {
    typedef typename MrType<CPLX>::T T;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int q2 = q * q;
    T* yp = reinterpret_cast<T*>(sm_raw);               // [q2][RC]
    T* U = yp + q2 * MR_RC;                             // [2][q][q][RC]
    float* Ss = reinterpret_cast<float*>(U + 2 * q2 * MR_RC);
    const int64_t pl = blockIdx.x;
    const int r0 = blockIdx.y * MR_RC;
    const int rc = R - r0 < MR_RC ? R - r0 : MR_RC;
    for (int i = threadIdx.x; i < 2 * q2; i += blockDim.x) Ss[i] = S[i];
    for (int i = threadIdx.x; i < q2 * MR_RC; i += blockDim.x) {
        const int r = i % MR_RC, a = i / MR_RC;
        yp[i] = r < rc ? yh[((offL + pl) * q2 + a) * R + r0 + r] : mr_zero(T());
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * q2 * MR_RC; i += blockDim.x) {
        const int r = i % MR_RC, rest = i / MR_RC;
        const int cx = rest / q2, av = (rest % q2) / q, bu = rest % q;
        const float* Su = Ss + cx * q2;
        const T* v = yp + (av * q) * MR_RC + r;
        T acc = mr_zero(T());
        for (int au = 0; au < q; ++au) acc = mr_axpy(Su[au * q + bu], v[au * MR_RC], acc);
        U[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * q2 * MR_RC; i += blockDim.x) {
        const int r = i % MR_RC, rest = i / MR_RC;
        const int c = rest / q2, bv = (rest % q2) / q, bu = rest % q;
        if (r >= rc) continue;
        const float* Sv = Ss + (c >> 1) * q2;
        const T* u = U + ((c & 1) * q2 + bu) * MR_RC + r;
        T acc = mr_zero(T());
        for (int av = 0; av < q; ++av) acc = mr_axpy(Sv[av * q + bv], u[av * q * MR_RC], acc);
        T* o = yh + ((offL1 + 4 * pl + c) * q2 + bv * q + bu) * R + r0 + r;
        if constexpr (CPLX) *o = make_float2(o->x + acc.x, o->y + acc.y);
        else *o += acc;
    }
}

// B tiles: per cluster [RP][KAP] BF16 in the canonical no-swizzle K-major layout;
// column k < q2 is Re x^[k] (x^[k] for Laplace), q2 <= k < 2 q2 is Im x^[k - q2].
template <bool CPLX>
__global__ void mr_bpack_kernel(int R, int RP, int KAP, int64_t C, int q2, const typename MrType<CPLX>::T* __restrict__ xh,
                                __nv_bfloat16* __restrict__ xb) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= C * RP * KAP) return;
    int k = (int)(idx % KAP);
    int64_t rem = idx / KAP;
    int r = (int)(rem % RP);
    int64_t c = rem / RP;
    float v = 0.0f;
    if (r < R) {
        if constexpr (CPLX) {
            if (k < q2) v = xh[(c * q2 + k) * R + r].x;
            else if (k < 2 * q2) v = xh[(c * q2 + k - q2) * R + r].y;
        } else {
            if (k < q2) v = xh[(c * q2 + k) * R + r];
        }
    }
    int64_t off = c * (int64_t)RP * KAP + ((int64_t)((r >> 3) * (KAP >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7));
    xb[off] = __float2bfloat16(v);
}

// ---- tensor-core coupling ---------------------------------------------------------------
__device__ inline unsigned tsm(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ inline uint64_t umma_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ inline bool tc_wait(uint64_t* bar, unsigned parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(tsm(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Q > 0: compiled for q = Q (index arithmetic of the K generation by shifts and
// constants); Q = 0: q and KAP at run time.
template <bool CPLX, int Q>
__global__ void __launch_bounds__(544) mr_coupling_tc_kernel(
    const int32_t* __restrict__ rows, const int64_t* __restrict__ fptr, const int32_t* __restrict__ fsrc,
    const float4* __restrict__ geo, int q_rt, int R, int RP, int KAP_rt, int tcols, float kappa,
    const __nv_bfloat16* __restrict__ xb, typename MrType<CPLX>::T* __restrict__ yh, long long wait_limit,
    int* __restrict__ status) {
    constexpr int MAP = 128;
    const int q = Q > 0 ? Q : q_rt;
    const int KAP = Q > 0 ? (((CPLX ? 2 * Q * Q : Q * Q) + 15) & ~15) : KAP_rt;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* bfull = reinterpret_cast<uint64_t*>(smem);        // [2]
    uint64_t* mdone = bfull + 2;                                 // [2]
    uint64_t* afull = bfull + 4;                                 // [2]: 16 warp arrivals per A tile
    int* issued_sh = reinterpret_cast<int*>(smem + 76);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 64);
    int* flag = reinterpret_cast<int*>(smem + 72);
    float4* Xs = reinterpret_cast<float4*>(smem + 128);
    const int q2 = q * q;
    const size_t abytes = (size_t)MAP * KAP * 2, bbytes = (size_t)RP * KAP * 2;
    unsigned char* tiles = smem + 1024 * ((128 + (size_t)q2 * 16 + 1023) / 1024);
    // buffer b: A tile at tiles + b * abytes, B tile at tiles + 2 * abytes + b * bbytes
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;   // 544 threads: 16 generating warps + 1
    const int sigma = rows[blockIdx.x];
    const int64_t b0 = fptr[sigma];
    const int n = (int)(fptr[sigma + 1] - b0);
    const int K8 = KAP >> 3;
    if (t == 0) {
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tsm(&bfull[i])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tsm(&mdone[i])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 16;" ::"r"(tsm(&afull[i])) : "memory");
        }
        *flag = 0;
        *issued_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tsm(tslot)), "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = t; i < q2; i += blockDim.x) {
        float4 g = geo[(int64_t)sigma * q2 + i];
        g.w *= 0.07957747154594767f;   // k / (4 pi)
        Xs[i] = g;
    }
    // padding rows / columns of both A buffers stay zero
    for (size_t i = t; i < 2 * abytes / 16; i += blockDim.x) reinterpret_cast<uint4*>(tiles)[i] = make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(RP >> 3) << 17) | ((uint32_t)(MAP >> 4) << 24);
    // Warps 0..15 generate the A tiles, warp 16 (lane 0) issues the moments' copy
    // and the MMAs.  No CTA barrier inside the loops: a generating thread waits by
    // itself until the MMAs of block i - 2 have released buffer i & 1, each warp
    // announces its part of the A tile on afull, and the issuing lane waits for
    // afull and for the copy (bfull).  A failed (bounded) wait raises the shared
    // flag, which every loop checks at the top of each block.
    volatile int* vflag = flag;
    int issued = 0;          // blocks whose MMAs were committed (issuing lane)
    bool failed = false;
    if (warp < 16) {
        for (int i = 0; i < n; ++i) {
            const int buf = i & 1;
            if (*vflag) { failed = true; break; }
            if (i >= 2 && !tc_wait(&mdone[buf], (unsigned)(((i - 2) >> 1) & 1), wait_limit)) {
                atomicOr(flag, 1);
                failed = true;
                break;
            }
            const int tau = fsrc[b0 + i];
            // A tile: the coupling block in FP32, stored as BF16.  A warp fills one
            // 8 x 8 core matrix per step (lane -> row lane / 4, columns 2 (lane % 4)
            // and +1) with packed 4-byte stores: 128 contiguous bytes, no bank conflicts.
            __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(tiles + buf * abytes);
            const float4* Y = geo + (int64_t)tau * q2;
            const int q8 = (q2 + 7) >> 3;
            // quadrant offsets of the real form when q2 is a multiple of 8
            const int offR = (q2 >> 3) * 64, offD = (q2 >> 3) * K8 * 64;
            const bool aligned8 = (q2 & 7) == 0;
            // 512 threads: 16 warps; with q fixed the trip count is known and the
            // loop unrolls, so a warp keeps several core matrices' SFU work in flight
    #pragma unroll
            for (int cm = warp; cm < q8 * q8; cm += 16) {
                const int ca = cm / q8, cb = cm - ca * q8;
                const int a = 8 * ca + (lane >> 2), b = 8 * cb + 2 * (lane & 3);
                if (a >= q2 || b >= q2) continue;   // q2 is even, so b + 1 < q2 as well
                const float4 X = Xs[a];
                float wr[2], wi[2];
    #pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const float4 Yb = Y[b + u];
                    const float d0 = X.x - Yb.x, d1 = X.y - Yb.y, d2 = X.z - Yb.z;
                    const float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
                    const float rinv = rsqrtf(r2);
                    const float w = X.w * Yb.w * rinv;          // X.w holds k / (4 pi)
                    if constexpr (CPLX) {
                        // phase reduced to [-pi, pi] first (the hardware sine and
                        // cosine are accurate on that interval only)
                        float ph = kappa * (r2 * rinv);
                        ph = fmaf(-6.283185307179586f, rintf(ph * 0.15915494309189535f), ph);
                        float sn, cs;
                        __sincosf(ph, &sn, &cs);
                        wr[u] = w * cs;
                        wi[u] = w * sn;
                    } else {
                        wr[u] = w;
                        wi[u] = 0.0f;
                    }
                }
                const int base = (ca * K8 + (b >> 3)) * 64 + (a & 7) * 8 + (b & 7);
                const __nv_bfloat162 kr = __floats2bfloat162_rn(wr[0], wr[1]);
                reinterpret_cast<__nv_bfloat162*>(A + base)[0] = kr;
                if constexpr (CPLX) {
                    const __nv_bfloat162 mki = __floats2bfloat162_rn(-wi[0], -wi[1]);
                    const __nv_bfloat162 ki = __floats2bfloat162_rn(wi[0], wi[1]);
                    if (aligned8) {
                        reinterpret_cast<__nv_bfloat162*>(A + base + offR)[0] = mki;
                        reinterpret_cast<__nv_bfloat162*>(A + base + offD)[0] = ki;
                        reinterpret_cast<__nv_bfloat162*>(A + base + offD + offR)[0] = kr;
                    } else {
                        auto at = [&](int m, int k) -> __nv_bfloat162* {
                            return reinterpret_cast<__nv_bfloat162*>(A + ((m >> 3) * K8 + (k >> 3)) * 64 + (m & 7) * 8 +
                                                                     (k & 7));
                        };
                        *at(a, b + q2) = mki;
                        *at(a + q2, b) = ki;
                        *at(a + q2, b + q2) = kr;
                    }
                }
            }
            // this warp's part of the A tile is written: make it visible to the
            // tensor core (async proxy) and announce it
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tsm(&afull[buf])) : "memory");
        }
    } else if (lane == 0) {
        for (int i = 0; i < n; ++i) {
            const int buf = i & 1;
            if (*vflag) { failed = true; break; }
            if (i >= 2 && !tc_wait(&mdone[buf], (unsigned)(((i - 2) >> 1) & 1), wait_limit)) {
                atomicOr(flag, 1);
                failed = true;
                break;
            }
            const int tau = fsrc[b0 + i];
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tsm(&bfull[buf])),
                         "r"((unsigned)bbytes)
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             tsm(tiles + 2 * abytes + buf * bbytes)),
                         "l"(xb + (int64_t)tau * RP * KAP), "r"((unsigned)bbytes), "r"(tsm(&bfull[buf]))
                         : "memory");
            const bool aok = tc_wait(&afull[buf], (unsigned)((i >> 1) & 1), wait_limit);
            const bool bok = aok && tc_wait(&bfull[buf], (unsigned)((i >> 1) & 1), wait_limit);
            if (!aok || !bok) {
                atomicOr(flag, 1);
                // the copy for this block may still land: wait for it before leaving
                tc_wait(&bfull[buf], (unsigned)((i >> 1) & 1), 1LL << 24);
                failed = true;
                break;
            }
            __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(tiles + buf * abytes);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int kk = 0; kk < KAP / 16; ++kk) {
                const uint64_t ad = umma_desc(tsm(A) + kk * 256, 128, K8 * 128);
                const uint64_t bd = umma_desc(tsm(tiles + 2 * abytes + buf * bbytes) + kk * 256, 128, K8 * 128);
                const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tsm(&mdone[buf]))
                         : "memory");
            issued = i + 1;
        }
    }
    if (t == 16 * 32) *issued_sh = issued;
    if (__syncthreads_or(failed)) failed = true;
    issued = *issued_sh;
    // wait for the last committed MMAs (bounded), then read the accumulator
    bool ok = true;
    if (issued > 0) {
        const int last = issued - 1;
        ok = tc_wait(&mdone[last & 1], (unsigned)((last >> 1) & 1), failed ? (1LL << 24) : wait_limit);
        if (issued > 1) {
            const int prev = issued - 2;
            tc_wait(&mdone[prev & 1], (unsigned)((prev >> 1) & 1), 1LL << 24);
        }
    }
    if (__syncthreads_or(!ok || failed)) {
        if (t == 0) atomicOr(status, 1);
    } else if (warp < 4) {
        // warps 0..3 own TMEM lane quarters 0..3
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = 32 * warp + lane;
        const int mvalid = CPLX ? 2 * q2 : q2;
        for (int c0 = 0; c0 < RP; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < mvalid) {
                for (int j = 0; j < 16; ++j) {
                    const int r = c0 + j;
                    if (r >= R) break;
                    const float val = __uint_as_float(v[j]);
                    if constexpr (CPLX) {
                        float* dst = reinterpret_cast<float*>(yh + ((int64_t)sigma * q2 + (row % q2)) * R + r);
                        dst[row < q2 ? 0 : 1] = val;
                    } else {
                        yh[((int64_t)sigma * q2 + row) * R + r] = val;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

// ---- stored BF16 coupling (IBEM_FP32_COUPLING_STORE, Helmholtz, q = 8) ----------------------
// Each far block is generated once at assembly, with the same FP32 formula as the
// generating kernel above, and kept as one 128 x 64 BF16 tile: rows a < 64 hold
// Re K[a][.], rows 64 + a hold Im K[a][.] (no-swizzle K-major layout, 16 KB).  An
// application packs the moments per cluster as [N = 2 RQ][64] BF16 (rows n < RQ
// the real parts of right-hand side n, rows RQ + n the imaginary parts), and one
// M = 128, N = 2 RQ MMA group per far block accumulates
// D = [Re K; Im K] [Re x^ | Im x^] in TMEM; the epilogue forms
// Re y^ = D[a][n] - D[64 + a][RQ + n], Im y^ = D[a][RQ + n] + D[64 + a][n].
// The kernel streams K (16 KB per block) and the moments by cp.async.bulk into
// a ring of NST stages: lane 0 of warp 0 issues the copies, lane 0 of warp 1
// the MMAs; all waits are bounded.  The depth (2, 3 or 4 stages: 3, 2 or 1
// resident CTAs per SM at 64 right-hand sides) is chosen by timing each once on
// the handle's first stored application.
constexpr int ST_Q2 = 64;            // q = 8
constexpr int ST_ABYTES = 128 * ST_Q2 * 2;

__device__ inline int st_tile_off(int m, int k) {   // element offset in a [rows][64] canonical tile
    return ((m >> 3) * 8 + (k >> 3)) * 64 + (m & 7) * 8 + (k & 7);
}

__global__ void mr_store_kernel(int64_t n_far, const int32_t* __restrict__ ftgt, const int32_t* __restrict__ fsrc,
                                const float4* __restrict__ geo, float kappa, __nv_bfloat16* __restrict__ K) {
    const int64_t blk = blockIdx.x;
    if (blk >= n_far) return;
    const float4* X = geo + (int64_t)ftgt[blk] * ST_Q2;
    const float4* Y = geo + (int64_t)fsrc[blk] * ST_Q2;
    __nv_bfloat16* T = K + blk * (128 * ST_Q2);
    for (int e = threadIdx.x; e < ST_Q2 * ST_Q2; e += blockDim.x) {
        const int a = e / ST_Q2, b = e % ST_Q2;
        const float4 x = X[a], y = Y[b];
        const float d0 = x.x - y.x, d1 = x.y - y.y, d2 = x.z - y.z;
        const float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
        const float rinv = rsqrtf(r2);
        const float w = (x.w * 0.07957747154594767f) * y.w * rinv;
        float ph = kappa * (r2 * rinv);
        ph = fmaf(-6.283185307179586f, rintf(ph * 0.15915494309189535f), ph);
        float sn, cs;
        __sincosf(ph, &sn, &cs);
        T[st_tile_off(a, b)] = __float2bfloat16(w * cs);
        T[st_tile_off(ST_Q2 + a, b)] = __float2bfloat16(w * sn);
    }
}

// moments x^ [C][64][R] (float2) -> per (chunk, cluster) [2 RQ][64] BF16 tiles
__global__ void mr_bpack_stored_kernel(int R, int RQ, int nch, int64_t C, const float2* __restrict__ xh,
                                       __nv_bfloat16* __restrict__ xb) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int N = 2 * RQ;
    if (idx >= (int64_t)nch * C * N * ST_Q2) return;
    const int k = (int)(idx % ST_Q2);
    int64_t rem = idx / ST_Q2;
    const int n = (int)(rem % N);
    rem /= N;
    const int64_t c = rem % C;
    const int ch = (int)(rem / C);
    const int r = ch * 64 + (n < RQ ? n : n - RQ);   // RQ <= 64
    float v = 0.0f;
    if (r < R) {
        const float2 x = xh[(c * ST_Q2 + k) * R + r];
        v = n < RQ ? x.x : x.y;
    }
    xb[((int64_t)ch * C + c) * N * ST_Q2 + st_tile_off(n, k)] = __float2bfloat16(v);
}

template <int ST_NST>
__global__ void __launch_bounds__(128) mr_coupling_stored_kernel(
    const int32_t* __restrict__ rows, const int64_t* __restrict__ fptr, const int32_t* __restrict__ fsrc,
    const __nv_bfloat16* __restrict__ Kst, const __nv_bfloat16* __restrict__ xb, int R, int RQ, int64_t C,
    int tcols, float2* __restrict__ yh, long long wait_limit, int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);          // [ST_NST]
    uint64_t* empty = full + ST_NST;                              // [ST_NST]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 128);
    int* flag = reinterpret_cast<int*>(smem + 136);
    int* counts = reinterpret_cast<int*>(smem + 144);             // blocks copied, blocks consumed
    const int N = 2 * RQ;
    const unsigned bbytes = (unsigned)N * ST_Q2 * 2;
    const size_t sbytes = ST_ABYTES + (size_t)bbytes;
    unsigned char* tiles = smem + 1024;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int sigma = rows[blockIdx.x];
    const int chunk = blockIdx.y;
    const int64_t b0 = fptr[sigma];
    const int n = (int)(fptr[sigma + 1] - b0);
    const __nv_bfloat16* xc = xb + (int64_t)chunk * C * N * ST_Q2;
    if (t == 0) {
        for (int i = 0; i < ST_NST; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tsm(&full[i])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tsm(&empty[i])) : "memory");
        }
        *flag = 0;
        counts[0] = counts[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tsm(tslot)), "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    int copied = 0, consumed = 0;
    volatile int* vflag = flag;
    bool failed = false;
    if (t == 0) {
        // producer: block i into stage i % ST_NST once the MMAs of block i - ST_NST are done
        for (int i = 0; i < n; ++i) {
            const int st = i % ST_NST;
            if (*vflag) { failed = true; break; }
            if (i >= ST_NST && !tc_wait(&empty[st], (unsigned)((i / ST_NST - 1) & 1), wait_limit)) {
                atomicOr(flag, 1);
                failed = true;
                break;
            }
            unsigned char* dst = tiles + st * sbytes;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tsm(&full[st])),
                         "r"((unsigned)ST_ABYTES + bbytes)
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             tsm(dst)),
                         "l"(Kst + (b0 + i) * (int64_t)(128 * ST_Q2)), "r"((unsigned)ST_ABYTES), "r"(tsm(&full[st]))
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             tsm(dst + ST_ABYTES)),
                         "l"(xc + (int64_t)fsrc[b0 + i] * N * ST_Q2), "r"(bbytes), "r"(tsm(&full[st]))
                         : "memory");
            copied = i + 1;
        }
        counts[0] = copied;
    } else if (t == 32) {
        // MMA issuer
        for (int i = 0; i < n; ++i) {
            const int st = i % ST_NST;
            if (*vflag) { failed = true; break; }
            if (!tc_wait(&full[st], (unsigned)((i / ST_NST) & 1), wait_limit)) {
                atomicOr(flag, 1);
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned char* src = tiles + st * sbytes;
            for (int kk = 0; kk < ST_Q2 / 16; ++kk) {
                const uint64_t ad = umma_desc(tsm(src) + kk * 256, 128, 8 * 128);
                const uint64_t bd = umma_desc(tsm(src + ST_ABYTES) + kk * 256, 128, 8 * 128);
                const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tsm(&empty[st]))
                         : "memory");
            consumed = i + 1;
        }
        counts[1] = consumed;
    }
    if (__syncthreads_or(failed)) failed = true;
    // the last committed MMA group completes the accumulator
    bool ok = !failed;
    if (n > 0 && ok) ok = tc_wait(&empty[(n - 1) % ST_NST], (unsigned)(((n - 1) / ST_NST) & 1), wait_limit);
    if (failed && t == 0) {
        // copies issued but not consumed land before the CTA leaves (bounded waits)
        for (int i = counts[1]; i < counts[0]; ++i) tc_wait(&full[i % ST_NST], (unsigned)((i / ST_NST) & 1), 1LL << 20);
        // MMAs committed but not waited for finish too
        if (counts[1] > 0) tc_wait(&empty[(counts[1] - 1) % ST_NST], (unsigned)(((counts[1] - 1) / ST_NST) & 1), 1LL << 20);
    }
    if (__syncthreads_or(!ok)) {
        if (t == 0) atomicOr(status, 1);
    } else if (n > 0) {
        // accumulator rows to shared memory (the ring is free), then combine
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float* S = reinterpret_cast<float*>(tiles);              // [128][N]
        const int row = 32 * warp + lane;
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            for (int j = 0; j < 16; ++j) S[row * N + c0 + j] = __uint_as_float(v[j]);
        }
        __syncthreads();
        const int r0 = chunk * 64;
        const int rc = R - r0 < 64 ? R - r0 : 64;
        for (int e = t; e < ST_Q2 * rc; e += blockDim.x) {
            const int a = e / rc, j = e % rc;
            const float yr = S[a * N + j] - S[(ST_Q2 + a) * N + RQ + j];
            const float yi = S[a * N + RQ + j] + S[(ST_Q2 + a) * N + j];
            yh[((int64_t)sigma * ST_Q2 + a) * R + r0 + j] = make_float2(yr, yi);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

template <int NST>
cudaError_t launch_stored_t(ibem_handle* h, unsigned nrows, int nch, const __nv_bfloat16* xb, int R, int RQ,
                            float2* yh) {
    int tcols = 32;
    while (tcols < 2 * RQ) tcols <<= 1;
    const size_t sm = 1024 + (size_t)NST * (ST_ABYTES + (size_t)2 * RQ * ST_Q2 * 2);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(mr_coupling_stored_kernel<NST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm)))
        return e;
    mr_coupling_stored_kernel<NST><<<dim3(nrows, nch), 128, sm, h->stream>>>(
        h->d_far_rows, h->d_far_ptr, h->d_far_src, reinterpret_cast<const __nv_bfloat16*>(h->d_Kbf), xb, R, RQ,
        h->P.C, tcols, yh, h->wait_limit, h->d_status);
    return cudaGetLastError();
}

cudaError_t launch_stored(ibem_handle* h, int nst, unsigned nrows, int nch, const __nv_bfloat16* xb, int R, int RQ,
                          float2* yh) {
    switch (nst) {
        case 2: return launch_stored_t<2>(h, nrows, nch, xb, R, RQ, yh);
        case 3: return launch_stored_t<3>(h, nrows, nch, xb, R, RQ, yh);
        default: return launch_stored_t<4>(h, nrows, nch, xb, R, RQ, yh);
    }
}

// ---- L2L, back-projection, near field, restriction ---------------------------------------
template <bool CPLX>
__global__ void mr_back_kernel(int R, int64_t E, int pp, int q, const float* __restrict__ M,
                               const typename MrType<CPLX>::T* __restrict__ yh, int64_t leaf_off,
                               typename MrType<CPLX>::T* __restrict__ ys) {
    typedef typename MrType<CPLX>::T T;
    const int q2 = q * q, nb = pp * pp;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= E * nb * R) return;
    int r = (int)(idx % R);
    int64_t rem = idx / R;
    int i = (int)(rem % nb);
    int64_t e = rem / nb;
    const int iu = i % pp, iv = i / pp;
    T acc = mr_zero(T());
    for (int av = 0; av < q; ++av)
        for (int au = 0; au < q; ++au)
            acc = mr_axpy(M[au * pp + iu] * M[av * pp + iv], yh[((leaf_off + e) * q2 + av * q + au) * R + r], acc);
    ys[idx] = acc;
}

// one CTA per target element; thread (i, r) over the row's near blocks
template <bool CPLX>
__global__ void mr_near_kernel(int R, int nb, const int64_t* __restrict__ nptr, const int32_t* __restrict__ nsrc,
                               const float* __restrict__ blocks, const typename MrType<CPLX>::T* __restrict__ xs,
                               typename MrType<CPLX>::T* __restrict__ ys) {
    typedef typename MrType<CPLX>::T T;
    const int64_t e = blockIdx.x;
    const int nbb = nb * nb;
    for (int o = threadIdx.x; o < nb * R; o += blockDim.x) {
        const int i = o / R, r = o % R;
        float ar = 0.0f, ai = 0.0f;
        for (int64_t k = nptr[e]; k < nptr[e + 1]; ++k) {
            const int64_t s = nsrc[k];
            for (int j = 0; j < nb; ++j) {
                const T x = xs[(s * nb + j) * R + r];
                if constexpr (CPLX) {
                    const float br = blocks[2 * (k * nbb + i * nb + j)], bi = blocks[2 * (k * nbb + i * nb + j) + 1];
                    ar = fmaf(br, x.x, fmaf(-bi, x.y, ar));
                    ai = fmaf(br, x.y, fmaf(bi, x.x, ai));
                } else {
                    ar = fmaf(blocks[k * nbb + i * nb + j], x, ar);
                }
            }
        }
        T* out = ys + (e * nb + i) * R + r;
        if constexpr (CPLX) *out = make_float2(out->x + ar, out->y + ai);
        else *out += ar;
    }
}

// Same product with one thread per right-hand side holding all NB rows of its
// element: the element's blocks pass through shared memory in chunks of KC
// (broadcast reads, 4 FMA per complex entry and load), each source value is
// loaded once per block (coalesced over the right-hand sides).  The sums run in
// the same order (blocks, then columns) as in mr_near_kernel.
template <bool CPLX, int NB>
__global__ void __launch_bounds__(256) mr_near_rows_kernel(int R, const int64_t* __restrict__ nptr,
                                                           const int32_t* __restrict__ nsrc,
                                                           const float* __restrict__ blocks,
                                                           const typename MrType<CPLX>::T* __restrict__ xs,
                                                           typename MrType<CPLX>::T* __restrict__ ys) {
    typedef typename MrType<CPLX>::T T;
    constexpr int CW = CPLX ? 2 : 1;
    constexpr int BF = NB * NB * CW;                             // floats per block
    constexpr int KC = (NB == 9 ? 32 : 8) * (CPLX ? 1 : 2);      // blocks per shared-memory chunk
    __shared__ float sb[KC * BF];
    __shared__ int ss[KC];
    const int64_t e = blockIdx.x;
    const int r = threadIdx.x;
    const bool act = r < R;
    float ar[NB], ai[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) ar[i] = ai[i] = 0.0f;
    const int64_t k0 = nptr[e], k1 = nptr[e + 1];
    for (int64_t kb = k0; kb < k1; kb += KC) {
        const int kc = (int)(k1 - kb < KC ? k1 - kb : KC);
        for (int i = threadIdx.x; i < kc * BF; i += blockDim.x) sb[i] = blocks[kb * BF + i];
        for (int i = threadIdx.x; i < kc; i += blockDim.x) ss[i] = nsrc[kb + i];
        __syncthreads();
        if (act) {
            for (int kk = 0; kk < kc; ++kk) {
                const int64_t s = ss[kk];
                T xv[NB];
#pragma unroll
                for (int j = 0; j < NB; ++j) xv[j] = xs[(s * NB + j) * R + r];
                const float* B = sb + kk * BF;
#pragma unroll
                for (int i = 0; i < NB; ++i) {
#pragma unroll
                    for (int j = 0; j < NB; ++j) {
                        if constexpr (CPLX) {
                            const float br = B[2 * (i * NB + j)], bi = B[2 * (i * NB + j) + 1];
                            ar[i] = fmaf(br, xv[j].x, fmaf(-bi, xv[j].y, ar[i]));
                            ai[i] = fmaf(br, xv[j].y, fmaf(bi, xv[j].x, ai[i]));
                        } else {
                            ar[i] = fmaf(B[i * NB + j], xv[j], ar[i]);
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    if (!act) return;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        T* out = ys + (e * NB + i) * R + r;
        if constexpr (CPLX) *out = make_float2(out->x + ar[i], out->y + ai[i]);
        else *out += ar[i];
    }
}

// y [R][N] (doubles, interleaved complex) = T y*
template <bool CPLX>
__global__ void mr_restrict_kernel(int R, int64_t N, int p, int ne1, const double* __restrict__ ext,
                                   const typename MrType<CPLX>::T* __restrict__ ys, double* __restrict__ y) {
    typedef typename MrType<CPLX>::T T;
    const int pp = p + 1, nb = pp * pp, n1 = ne1 + p;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R * N) return;
    int r = (int)(idx % R);
    int64_t dof = idx / R;
    int patch = (int)(dof / ((int64_t)n1 * n1));
    int rem = (int)(dof % ((int64_t)n1 * n1));
    int jv = rem / n1, ju = rem % n1;
    int64_t per = (int64_t)ne1 * ne1;
    float ar = 0.0f, ai = 0.0f;
    for (int iy = jv - p; iy <= jv; ++iy) {
        if (iy < 0 || iy >= ne1) continue;
        for (int ix = ju - p; ix <= ju; ++ix) {
            if (ix < 0 || ix >= ne1) continue;
            const int64_t e = patch * per + morton2(ix, iy);
            const double* cu = ext + ((int64_t)ix * pp + (ju - ix)) * pp;
            const double* cv = ext + ((int64_t)iy * pp + (jv - iy)) * pp;
            for (int iv = 0; iv < pp; ++iv)
                for (int iu = 0; iu < pp; ++iu) {
                    const float c = (float)cu[iu] * (float)cv[iv];
                    const T v = ys[(e * nb + iv * pp + iu) * R + r];
                    if constexpr (CPLX) {
                        ar += c * v.x;
                        ai += c * v.y;
                    } else {
                        ar += c * v;
                    }
                }
        }
    }
    if constexpr (CPLX) {
        y[2 * (r * N + dof)] = ar;
        y[2 * (r * N + dof) + 1] = ai;
    } else {
        y[r * N + dof] = ar;
    }
}

template <bool CPLX>
static cudaError_t mr_apply(ibem_handle* h, const double* x, double* y, int R) {
    typedef typename MrType<CPLX>::T T;
    Plan& P = h->P;
    cudaStream_t st = h->stream;
    cudaError_t e;
    const int T_ = 256;
    const int q2 = P.q2;
    const int RP = (R + 15) & ~15;
    const int KAP = ((CPLX ? 2 * q2 : q2) + 15) & ~15;
    // work space (grown on demand)
    const size_t need_t = (size_t)R * P.N, need_s = (size_t)R * P.Nstar, need_h = (size_t)R * P.C * (q2 > 0 ? q2 : 1);
    // moments as BF16 tiles: generated coupling [C][RP][KAP]; stored coupling
    // [nch][C][2 RQ][64] with chunks of 64 right-hand sides
    const bool stored = CPLX && h->d_Kbf != nullptr;
    const int RQ = ((R < 64 ? R : 64) + 7) & ~7, nch = (R + 63) / 64;
    size_t need_b = (size_t)P.C * RP * (KAP > 0 ? KAP : 16);
    if (stored) need_b = std::max(need_b, (size_t)nch * P.C * 2 * RQ * ST_Q2);
    const size_t bytes = sizeof(T) * (need_t + 2 * need_s + 2 * need_h) + 2 * need_b + 1024;
    if (bytes > h->mr_bytes) {
        cudaFree(h->d_mr);
        h->d_mr = nullptr;
        h->mr_bytes = 0;
        if ((e = cudaMalloc(&h->d_mr, bytes))) return e;
        h->mr_bytes = bytes;
    }
    T* xt = reinterpret_cast<T*>(h->d_mr);
    T* xs = xt + need_t;
    T* ys = xs + need_s;
    T* xh = ys + need_s;
    T* yh = xh + need_h;
    __nv_bfloat16* xb = reinterpret_cast<__nv_bfloat16*>(
        reinterpret_cast<unsigned char*>(h->d_mr) + (((sizeof(T) * (need_t + 2 * need_s + 2 * need_h)) + 255) / 256) * 256);
    {
        PhaseTimer pt(h, 0);
        mr_in_kernel<CPLX><<<nblk((int64_t)R * P.N, T_), T_, 0, st>>>(R, P.N, x, xt);
        mr_lift_kernel<CPLX><<<nblk(P.E * P.nb * R, T_), T_, 0, st>>>(R, P.E, P.p, P.ne1, h->d_ext, xt, xs);
        h->launches += 2;
    }
    if ((e = cudaMemsetAsync(ys, 0, need_s * sizeof(T), st))) return e;
    if (P.q > 0) {
        const int64_t leaf_off = P.level_off[P.m];
        {
            PhaseTimer pt(h, 1);
            mr_leaf_kernel<CPLX><<<nblk(P.E * q2 * R, T_), T_, 0, st>>>(R, P.E, P.pp, P.q, h->d_Mf, xs, leaf_off, xh);
            h->launches++;
            const size_t smm = (size_t)8 * q2 * MR_RC * sizeof(T) + 2 * q2 * sizeof(float);
            for (int L = P.m - 1; L >= 0; --L) {
                int64_t nL = P.level_off[L + 1] - P.level_off[L];
                mr_m2m_sep_kernel<CPLX><<<dim3((unsigned)nL, (R + MR_RC - 1) / MR_RC), 256, smm, st>>>(
                    R, P.level_off[L], P.level_off[L + 1], P.q, h->d_Sf, xh);
                h->launches++;
            }
        }
        if ((e = cudaMemsetAsync(yh, 0, need_h * sizeof(T), st))) return e;
        const unsigned nrows = (unsigned)h->far_rows.size();
        if (nrows > 0 && stored) {
            PhaseTimer pt(h, 2);
            mr_bpack_stored_kernel<<<nblk((int64_t)nch * P.C * 2 * RQ * ST_Q2, T_), T_, 0, st>>>(
                R, RQ, nch, P.C, reinterpret_cast<const float2*>(xh), xb);
            h->launches++;
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            if ((e = cudaStreamIsCapturing(st, &cap))) return e;
            if (h->st_nst == 0 && cap == cudaStreamCaptureStatusNone) {
                // first stored application: time each ring depth once (the kernel
                // overwrites its rows, so the extra runs change nothing)
                cudaEvent_t ev[2];
                if ((e = cudaEventCreate(&ev[0]))) return e;
                if ((e = cudaEventCreate(&ev[1]))) {
                    cudaEventDestroy(ev[0]);
                    return e;
                }
                float best = 1e30f;
                int pick = 4;
                for (int nst : {4, 3, 2}) {
                    if ((e = launch_stored(h, nst, nrows, nch, xb, R, RQ, reinterpret_cast<float2*>(yh)))) break;
                    cudaEventRecord(ev[0], st);
                    if ((e = launch_stored(h, nst, nrows, nch, xb, R, RQ, reinterpret_cast<float2*>(yh)))) break;
                    cudaEventRecord(ev[1], st);
                    if ((e = cudaEventSynchronize(ev[1]))) break;
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, ev[0], ev[1]);
                    if (ms < best) {
                        best = ms;
                        pick = nst;
                    }
                }
                cudaEventDestroy(ev[0]);
                cudaEventDestroy(ev[1]);
                if (e) return e;
                h->st_nst = pick;
            }
            if ((e = launch_stored(h, h->st_nst ? h->st_nst : 4, nrows, nch, xb, R, RQ,
                                   reinterpret_cast<float2*>(yh))))
                return e;
            h->launches++;
        } else if (nrows > 0) {
            PhaseTimer pt(h, 2);
            mr_bpack_kernel<CPLX><<<nblk((int64_t)P.C * RP * KAP, T_), T_, 0, st>>>(R, RP, KAP, P.C, q2, xh, xb);
            int tcols = 32;
            while (tcols < RP) tcols <<= 1;
            const size_t sm = 1024 * ((128 + (size_t)q2 * 16 + 1023) / 1024) + 2 * (size_t)128 * KAP * 2 +
                              2 * (size_t)RP * KAP * 2;
            auto kern = P.q == 8 ? mr_coupling_tc_kernel<CPLX, 8>
                                 : (P.q == 6 ? mr_coupling_tc_kernel<CPLX, 6> : mr_coupling_tc_kernel<CPLX, 0>);
            if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
            kern<<<nrows, 544, sm, st>>>(h->d_far_rows, h->d_far_ptr, h->d_far_src,
                                         reinterpret_cast<const float4*>(h->d_igeo32), P.q, R, RP, KAP, tcols,
                                         (float)P.prm.kappa, xb, yh, h->wait_limit, h->d_status);
            h->launches += 2;
        }
        PhaseTimer pt(h, 3);
        const size_t sml = (size_t)3 * q2 * MR_RC * sizeof(T) + 2 * q2 * sizeof(float);
        for (int L = 0; L < P.m; ++L) {
            int64_t nL = P.level_off[L + 1] - P.level_off[L];
            mr_l2l_sep_kernel<CPLX><<<dim3((unsigned)nL, (R + MR_RC - 1) / MR_RC), 256, sml, st>>>(
                R, P.level_off[L], P.level_off[L + 1], P.q, h->d_Sf, yh);
            h->launches++;
        }
        mr_back_kernel<CPLX><<<nblk(P.E * P.nb * R, T_), T_, 0, st>>>(R, P.E, P.pp, P.q, h->d_Mf, yh, leaf_off, ys);
        h->launches++;
    }
    int nthreads = P.nb * R < 512 ? ((P.nb * R + 31) / 32) * 32 : 512;
    {
        PhaseTimer pt(h, 4);
        const int tr = ((R + 31) / 32) * 32;
        if (P.nb == 9)
            mr_near_rows_kernel<CPLX, 9><<<(unsigned)P.E, tr, 0, st>>>(R, h->d_near_ptr, h->d_near_src, h->d_near32,
                                                                       xs, ys);
        else if (P.nb == 16)
            mr_near_rows_kernel<CPLX, 16><<<(unsigned)P.E, tr, 0, st>>>(R, h->d_near_ptr, h->d_near_src, h->d_near32,
                                                                        xs, ys);
        else
            mr_near_kernel<CPLX><<<(unsigned)P.E, nthreads, 0, st>>>(R, P.nb, h->d_near_ptr, h->d_near_src,
                                                                     h->d_near32, xs, ys);
    }
    {
        PhaseTimer pt(h, 5);
        mr_restrict_kernel<CPLX><<<nblk((int64_t)R * P.N, T_), T_, 0, st>>>(R, P.N, P.p, P.ne1, h->d_ext, ys, y);
    }
    h->launches += 2;
    return cudaGetLastError();
}

bool mr_store_possible(const ibem_handle* h) { return h->helm && h->P.q2 == ST_Q2 && h->P.n_far > 0; }

cudaError_t mr_store_coupling(ibem_handle* h) {
    const Plan& P = h->P;
    mr_store_kernel<<<(unsigned)P.n_far, 256, 0, h->stream>>>(P.n_far, h->d_far_tgt, h->d_far_src,
                                                              reinterpret_cast<const float4*>(h->d_igeo32),
                                                              (float)P.prm.kappa,
                                                              reinterpret_cast<__nv_bfloat16*>(h->d_Kbf));
    return cudaGetLastError();
}

bool mr_supported(const ibem_handle* h, int nrhs) {
    const Plan& P = h->P;
    if (nrhs < 16 || nrhs > 256) return false;
    if (P.q == 0) return true;
    // even q: the A tile is written in aligned pairs of columns
    return (P.q % 2 == 0) && (h->helm ? 2 * P.q2 : P.q2) <= 128;
}

cudaError_t apply_operator_mrhs(ibem_handle* h, const double* x, double* y, int nrhs) {
    h->applications++;
    return h->helm ? mr_apply<true>(h, x, y, nrhs) : mr_apply<false>(h, x, y, nrhs);
}

}  // namespace ibem
