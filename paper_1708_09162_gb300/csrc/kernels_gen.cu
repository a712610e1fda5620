// FP64-accurate Helmholtz coupling for many right-hand sides, generated on the
// fly (Sec. 4.2: on a far block the coupling is y^_s += K_st x^_t with
// K_st[a][b] = k(z_a) k(z_b) e^{i kappa r} / (4 pi r), r = |F(z_a) - F(z_b)|).
//
// GB300 issues FP64 FMA at 1/64 of the FP32 rate, so K is generated and applied
// in double-float arithmetic (a value is an unevaluated sum h + l of two floats,
// about 48 significant bits) on the FP32 pipe, and every generated block is
// applied to all right-hand sides of the CTA's chunk before the next one is
// generated: the generation cost is shared by up to 64 right-hand sides.
//
// Kernel value in double-float: coordinates and surface measures of the
// interpolation points are tabulated as float pairs; d = X - Y, r^2 and r by one
// correction of the correctly rounded float square root; 1/r by one Newton step
// from the correctly rounded reciprocal; the phase theta = kappa r is reduced
// as theta = n c + t with c = 2 pi / 2048 split into four parts (Cody and
// Waite; c_1..c_3 with 9 significant bits), so that the products n c_1, n c_2,
// n c_3 are exact for n < 2^15 (theta < 100); e^{i theta} =
// e^{i n c} e^{i t} with e^{i n c} from a table of 2048 double-float values of
// cos and sin (computed on the host in extended precision) and e^{i t} from its
// Taylor series, |t| <= c / 2: sin t = t - t^3/6 + t^5/120, cos t = 1 - t^2/2 +
// t^4/24 (the next terms are below 1e-16).  The row factor k(z_a) / (4 pi) is
// applied in FP64 when the row is written.
//
// One CTA per (target cluster sigma, chunk of RC right-hand sides).  For each far
// block (sigma, tau): the source cluster's point table and its moments x^_tau
// (RC columns, complex double-float) arrive by one cp.async.bulk each, double
// buffered; the CTA generates K[a][b] into shared memory, then thread (rows a,
// a + 1; columns r .. r + 3; b-split) accumulates the products with exact
// FP32 products and compensated (TwoSum) accumulation.  The sums stay in
// registers over the whole far row (no atomics, fixed order: deterministic).
// All waits are bounded.
//
// The same kernel values can instead be contracted on the tensor cores
// (helm_coupling_sliced_kernel, IBEM_COUPLING_SLICED): kernel values and
// moments are split into BF16 digit slices whose pairwise products the FP32
// accumulation of tcgen05.mma keeps exactly, and the exact integer sums are
// recombined in double-float (see the description above that kernel).
#include <cuda_bf16.h>

#include <cmath>

#include "ibem_internal.cuh"

namespace ibem {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

namespace {

constexpr int GEN_THREADS = 512;
constexpr int GEN_TABLE = 2048;     // entries of the e^{i n c} table

struct df {
    float h, l;
};

// s + e = a + b exactly, for |a| >= |b| (Dekker)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}
// s + e = a + b exactly (Knuth)
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df df_add(df x, df y) {
    const df s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, s.l + (x.l + y.l));
}
__device__ __forceinline__ df df_neg(df x) { return {-x.h, -x.l}; }
__device__ __forceinline__ df df_mul(df x, df y) {
    const float p = x.h * y.h;
    float e = fmaf(x.h, y.h, -p);
    e = fmaf(x.h, y.l, fmaf(x.l, y.h, e));
    return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_sqr(df x) {
    const float p = x.h * x.h;
    float e = fmaf(x.h, x.h, -p);
    e = fmaf(2.0f * x.h, x.l, e);
    return fast_two_sum(p, e);
}

// acc (hi, lo) += a * b for double-float a, b: exact leading product, its
// rounding error and the cross terms into lo, TwoSum of the leading parts
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float& hi, float& lo) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, fmaf(al, bh, e));
    const float t = hi + p;
    const float z = t - hi;
    const float err = (hi - (t - z)) + (p - z);
    hi = t;
    lo += err + e;
}

struct GenConst {
    float kh, kl;               // kappa as double-float
    float inv_c;                // 1 / c, c = 2 pi / GEN_TABLE
    float c1, c2, c3, c4;       // c = c1 + c2 + c3 + c4; c1..c3 with 9 significant bits
};

// K'[b] = k(z_b) e^{i kappa r} / r in double-float (re, im): X, Y = (x, y, z, k)
// hi and lo parts of the two interpolation points
__device__ __forceinline__ void gen_entry(const float4 Xh, const float4 Xl, const float4 Yh, const float4 Yl,
                                          const GenConst& g, const float4* __restrict__ trig, df& kre, df& kim) {
    const df d0 = df_add({Xh.x, Xl.x}, {-Yh.x, -Yl.x});
    const df d1 = df_add({Xh.y, Xl.y}, {-Yh.y, -Yl.y});
    const df d2 = df_add({Xh.z, Xl.z}, {-Yh.z, -Yl.z});
    const df r2 = df_add(df_add(df_sqr(d0), df_sqr(d1)), df_sqr(d2));
    // r = sqrt(r2): s correctly rounded, then one correction (r2 - s^2) / (2 s)
    const float s = sqrtf(r2.h);
    const float ss = s * s;
    const float se = fmaf(s, s, -ss);
    const float corr = (((r2.h - ss) - se) + r2.l) * (0.5f * rsqrtf(r2.h));
    const df r = fast_two_sum(s, corr);
    // 1 / r: q0 correctly rounded, one Newton step on the exact residual
    const float q0 = __frcp_rn(r.h);
    const float res = fmaf(-r.l, q0, fmaf(-r.h, q0, 1.0f));
    const df inv = fast_two_sum(q0, q0 * res);
    const df amp = df_mul({Yh.w, Yl.w}, inv);
    // theta = kappa r = n c + t: n c1, n c2, n c3 are exact (n < 2^15), the
    // large differences are formed by exact two-sums
    const df th = df_mul({g.kh, g.kl}, r);
    const float n = rintf(th.h * g.inv_c);
    const df s1 = two_sum(th.h, -n * g.c1);
    const df v = two_sum(s1.h, -n * g.c2);
    const df w = two_sum(th.l, -n * g.c3);
    df t = df_add(v, w);
    t = fast_two_sum(t.h, t.l + fmaf(-n, g.c4, s1.l));
    // e^{i t}: Taylor series in t, |t| <= c / 2
    const float t2 = t.h * t.h;
    const float t3 = t2 * t.h;
    const df sn = df_add(t, {fmaf(t3, t2 * (1.0f / 120.0f), -t3 * (1.0f / 6.0f)), 0.0f});
    const float p = t2;
    const float pe = fmaf(t.h, t.h, -p);
    const df c0 = two_sum(1.0f, -0.5f * p);
    const df cs = fast_two_sum(c0.h, c0.l - fmaf(0.5f, pe, t.h * t.l) + t2 * t2 * (1.0f / 24.0f));
    // e^{i n c} from the table, times the amplitude, times e^{i t}
    const float4 e = trig[((int)n) & (GEN_TABLE - 1)];
    const df ar = df_mul(amp, {e.x, e.y}), ai = df_mul(amp, {e.z, e.w});
    kre = df_add(df_mul(ar, cs), df_neg(df_mul(ai, sn)));
    kim = df_add(df_mul(ai, cs), df_mul(ar, sn));
}

__device__ inline unsigned gsm(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ inline bool gen_wait(uint64_t* bar, unsigned parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(gsm(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ inline void gen_bulk(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     gsm(dst)),
                 "l"(src), "r"(bytes), "r"(gsm(bar))
                 : "memory");
}

// Shared memory: [0, 128) two mbarriers; point table of sigma [q2][2] float4;
// two stages of (point table of tau [q2][2] float4, moments [q2][RC] float4);
// K [q2][q2 + 1] float4 (one float4 of padding per row against bank conflicts),
// at least large enough for the final reduction of the b-splits
// ((splits - 1) * tiles * 8 float4 <= GEN_THREADS * 8 float4).
inline size_t gen_smem_bytes(int q2, int RC) {
    size_t kb = (size_t)q2 * (q2 + 1) * 16, rb = (size_t)GEN_THREADS * 8 * 16;
    return 128 + (size_t)q2 * 32 + 2 * ((size_t)q2 * 32 + (size_t)q2 * RC * 16) + (kb > rb ? kb : rb);
}

// pts: [C][q2][2] float4 = ((x, y, z, k) hi, (x, y, z, k) lo); xg: [nch][C][q2][RC]
// float4 (re_h, re_l, im_h, im_l); yh: split layout [2R][C][q2] doubles.
template <int RC>
__global__ void __launch_bounds__(GEN_THREADS, 1)
    helm_coupling_gen_kernel(const int32_t* __restrict__ rows, const int64_t* __restrict__ fptr,
                             const int32_t* __restrict__ fsrc, const float4* __restrict__ pts,
                             const double* __restrict__ igeo, const float4* __restrict__ trig, GenConst g, int q2,
                             int R, int64_t C, const float4* __restrict__ xg, double* __restrict__ yh,
                             long long wait_limit, int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    float4* Xs = reinterpret_cast<float4*>(smem + 128);
    float4* stage0 = Xs + 2 * q2;
    const int sel = 2 * q2 + q2 * RC;                    // float4 per stage
    float4* Ks = stage0 + 2 * sel;
    const int kst = q2 + 1;                              // K row stride (float4)
    const int sigma = rows[blockIdx.x];
    const int chunk = blockIdx.y;
    const int64_t b0 = fptr[sigma];
    const int n = (int)(fptr[sigma + 1] - b0);
    const int tid = threadIdx.x;
    const float4* xc = xg + (int64_t)chunk * C * q2 * RC;
    const unsigned pbytes = (unsigned)q2 * 32u, xbytes = (unsigned)q2 * RC * 16u;
    // application tiles: rows (2 ap, 2 ap + 1), columns 4 rq .. 4 rq + 3, b-split
    constexpr int RQ = RC / 4;
    const int ntile = ((q2 + 1) / 2) * RQ;
    int S = GEN_THREADS / ntile;
    S = S >= 8 ? 8 : (S >= 4 ? 4 : (S >= 2 ? 2 : 1));
    const int tile = tid % ntile, split = tid / ntile;
    const bool act = split < S;
    const int a0 = 2 * (tile / RQ), r0 = 4 * (tile % RQ);
    const bool row1 = a0 + 1 < q2;
    for (int i = tid; i < 2 * q2; i += blockDim.x) Xs[i] = pts[(int64_t)sigma * q2 * 2 + i];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(gsm(&full[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(gsm(&full[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int i = 0; i < 2 && i < n; ++i) {
            const int tau = fsrc[b0 + i];
            float4* st = stage0 + i * sel;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(gsm(&full[i])),
                         "r"(pbytes + xbytes)
                         : "memory");
            gen_bulk(st, pts + (int64_t)tau * q2 * 2, pbytes, &full[i]);
            gen_bulk(st + 2 * q2, xc + (int64_t)tau * q2 * RC, xbytes, &full[i]);
        }
    }
    __syncthreads();
    float acc[2][4][4];   // [row][column][re_h, re_l, im_h, im_l]
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.0f;
    bool failed = false;
    int i = 0;
    for (; i < n; ++i) {
        const int buf = i & 1;
        const bool ok = gen_wait(&full[buf], (unsigned)((i >> 1) & 1), wait_limit);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        const float4* Ys = stage0 + buf * sel;
        const float4* xs = Ys + 2 * q2;
        // generate K'[a][b] = k_b e^{i kappa r} / r
        for (int e = tid; e < q2 * q2; e += blockDim.x) {
            const int a = e / q2, b = e - a * q2;
            df kr, ki;
            gen_entry(Xs[2 * a], Xs[2 * a + 1], Ys[2 * b], Ys[2 * b + 1], g, trig, kr, ki);
            Ks[a * kst + b] = make_float4(kr.h, kr.l, ki.h, ki.l);
        }
        __syncthreads();
        // the stage of block i - 1 is free again: fetch block i + 1 into it
        if (tid == 0 && i >= 1 && i + 1 < n) {
            const int tau = fsrc[b0 + i + 1];
            float4* st = stage0 + ((i + 1) & 1) * sel;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(gsm(&full[(i + 1) & 1])),
                         "r"(pbytes + xbytes)
                         : "memory");
            gen_bulk(st, pts + (int64_t)tau * q2 * 2, pbytes, &full[(i + 1) & 1]);
            gen_bulk(st + 2 * q2, xc + (int64_t)tau * q2 * RC, xbytes, &full[(i + 1) & 1]);
        }
        if (act) {
            for (int b = split; b < q2; b += S) {
                const float4 k0 = Ks[a0 * kst + b];
                const float4 k1 = row1 ? Ks[(a0 + 1) * kst + b] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4* xr = xs + b * RC + r0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float4 x = xr[j];
                    // (Kr + i Ki)(xr + i xi) = (Kr xr - Ki xi) + i (Kr xi + Ki xr)
                    df_mac(k0.x, k0.y, x.x, x.y, acc[0][j][0], acc[0][j][1]);
                    df_mac(-k0.z, -k0.w, x.z, x.w, acc[0][j][0], acc[0][j][1]);
                    df_mac(k0.x, k0.y, x.z, x.w, acc[0][j][2], acc[0][j][3]);
                    df_mac(k0.z, k0.w, x.x, x.y, acc[0][j][2], acc[0][j][3]);
                    df_mac(k1.x, k1.y, x.x, x.y, acc[1][j][0], acc[1][j][1]);
                    df_mac(-k1.z, -k1.w, x.z, x.w, acc[1][j][0], acc[1][j][1]);
                    df_mac(k1.x, k1.y, x.z, x.w, acc[1][j][2], acc[1][j][3]);
                    df_mac(k1.z, k1.w, x.x, x.y, acc[1][j][2], acc[1][j][3]);
                }
            }
            // keep the low parts small against the leading ones
#pragma unroll
            for (int ii = 0; ii < 2; ++ii)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const df a = fast_two_sum(acc[ii][j][0], acc[ii][j][1]);
                    const df c = fast_two_sum(acc[ii][j][2], acc[ii][j][3]);
                    acc[ii][j][0] = a.h;
                    acc[ii][j][1] = a.l;
                    acc[ii][j][2] = c.h;
                    acc[ii][j][3] = c.l;
                }
        }
        __syncthreads();
    }
    if (failed) {
        if (tid == 0) {
            atomicOr(status, 1);
            // copies of blocks i and i + 1 may still be in flight
            for (int j = i; j < n && j < i + 2; ++j) gen_wait(&full[j & 1], (unsigned)((j >> 1) & 1), 1LL << 24);
        }
        __syncthreads();
        return;
    }
    // reduce the b-splits through shared memory (the K area is free now), then
    // write the row: y^_sigma[a][r] = k_a / (4 pi) * sum, in FP64
    float4* red = Ks;
    if (act && split > 0)
#pragma unroll
        for (int ii = 0; ii < 2; ++ii)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                red[((split - 1) * ntile + tile) * 8 + ii * 4 + j] =
                    make_float4(acc[ii][j][0], acc[ii][j][1], acc[ii][j][2], acc[ii][j][3]);
    __syncthreads();
    if (act && split == 0) {
        for (int s2 = 1; s2 < S; ++s2)
#pragma unroll
            for (int ii = 0; ii < 2; ++ii)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float4 v = red[((s2 - 1) * ntile + tile) * 8 + ii * 4 + j];
                    const df a = df_add({acc[ii][j][0], acc[ii][j][1]}, {v.x, v.y});
                    const df c = df_add({acc[ii][j][2], acc[ii][j][3]}, {v.z, v.w});
                    acc[ii][j][0] = a.h;
                    acc[ii][j][1] = a.l;
                    acc[ii][j][2] = c.h;
                    acc[ii][j][3] = c.l;
                }
#pragma unroll
        for (int ii = 0; ii < 2; ++ii) {
            const int a = a0 + ii;
            if (a >= q2) continue;
            const double ka = igeo[4 * ((int64_t)sigma * q2 + a) + 3] / (4.0 * IBEM_PI);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = chunk * RC + r0 + j;
                if (r >= R) continue;
                const double re = ((double)acc[ii][j][0] + (double)acc[ii][j][1]) * ka;
                const double im = ((double)acc[ii][j][2] + (double)acc[ii][j][3]) * ka;
                yh[((int64_t)(2 * r) * C + sigma) * q2 + a] = re;
                yh[((int64_t)(2 * r + 1) * C + sigma) * q2 + a] = im;
            }
        }
    }
}

// moments of the split layout [2R][C][q2] -> chunked double-float complex
// [nch][C][q2][RC] (zero columns beyond R)
__global__ void gen_split_kernel(int R, int RC, int nch, int64_t C, int q2, const double* __restrict__ xh,
                                 float4* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)nch * C * q2 * RC;
    if (idx >= total) return;
    const int rc = (int)(idx % RC);
    int64_t rem = idx / RC;
    const int b = (int)(rem % q2);
    rem /= q2;
    const int64_t c = rem % C;
    const int ch = (int)(rem / C);
    const int r = ch * RC + rc;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < R) {
        const double vr = xh[((int64_t)(2 * r) * C + c) * q2 + b];
        const double vi = xh[((int64_t)(2 * r + 1) * C + c) * q2 + b];
        const float rh = (float)vr, ih = (float)vi;
        v = make_float4(rh, (float)(vr - (double)rh), ih, (float)(vi - (double)ih));
    }
    out[idx] = v;
}

// point table [C][q2][2] float4 from the FP64 table [C][q2][4] (x, y, z, k)
__global__ void gen_points_kernel(int64_t n, const double* __restrict__ igeo, float4* __restrict__ pts) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float hi[4], lo[4];
    for (int k = 0; k < 4; ++k) {
        const double v = igeo[4 * i + k];
        hi[k] = (float)v;
        lo[k] = (float)(v - (double)hi[k]);
    }
    pts[2 * i] = make_float4(hi[0], hi[1], hi[2], hi[3]);
    pts[2 * i + 1] = make_float4(lo[0], lo[1], lo[2], lo[3]);
}

// float with at most `bits` significant bits nearest to v (for the Cody-Waite split)
// ---- FP64-accurate coupling on the tensor cores: digit slices ---------------------------
// An Ozaki-type splitting: every operand is written as a power of two times a
// sum of SL_S signed digits, v = 2^E sum_s d_s 2^{-7 - 8 s} with |d_s| <= 128
// (integers, exact in BF16), so that a product of two digit slices is an exact
// integer matrix product.  With K = 64 terms a slice pair sums to at most 2^20
// and a level k = s + t holds at most 6 pairs, below 2^23, which the FP32
// accumulation of tcgen05.mma kind::f16 keeps exactly (measured for sums below
// 2^24), so the 6 accumulators D_k = sum_{s + t = k} A_s B_t^T are exact and
//     K x = 2^{E + F - 14} sum_k 2^{-8 k} D_k
// up to the omitted levels k >= 6 (below 2^-45 of the block's scale) and the
// digits beyond the sixth (47 bits).  K'
// (k(z_b) e^{i kappa r} / r) is generated per far block in double-float as in
// helm_coupling_gen_kernel; E is per block (its largest |K'|), F per source
// cluster and column of moments.  Real form: A = [Re K'; Im K'] (128 x 64),
// B columns n < 32 the real, 32 + n the imaginary parts of 32 right-hand
// sides; Re y = D[a][n] - D[64 + a][32 + n], Im y = D[a][32 + n] + D[64 + a][n].
constexpr int SL_S = 6;                        // digit slices per operand
constexpr int SL_N = 64;                       // B rows per chunk: 32 complex right-hand sides
constexpr int SL_RQ = SL_N / 2;
constexpr int SL_Q2 = 64;                      // q = 8
constexpr int SL_THREADS = 512;
constexpr int SL_ATILE = 128 * SL_Q2 * 2;      // bytes of one A slice
constexpr int SL_BTILE = SL_N * SL_Q2 * 2;     // bytes of one B slice
constexpr int SL_BSTAGE = SL_S * SL_BTILE;     // all B slices of one source cluster
// shared memory map (bytes)
constexpr int SL_OFF_BAR = 0;                  // fullY[2], fullB, done: 4 mbarriers
constexpr int SL_OFF_TSLOT = 64;
constexpr int SL_OFF_RED = 128;                // [16] warp maxima
constexpr int SL_OFF_SC = 256;                 // [2][65] int: F of the columns, then E
constexpr int SL_OFF_F = 1024;                 // [2][64] int: column exponents of the staged source
constexpr int SL_OFF_X = 1536;                 // [64][2] float4 target points
constexpr int SL_OFF_Y = SL_OFF_X + 2048;      // [2][64][2] float4 source points
constexpr int SL_KST = 65;                     // row stride (float4) of the kernel-value staging buffer
constexpr int SL_OFF_K = 8192;                 // [64][SL_KST] float4: K' (re_h, re_l, im_h, im_l)
constexpr int SL_OFF_A = SL_OFF_K + SL_Q2 * SL_KST * 16;   // [SL_S] A slices (1024-aligned)
constexpr int SL_OFF_B = SL_OFF_A + SL_S * SL_ATILE;       // the SL_S B slices of one source cluster
constexpr int SL_SMEM = SL_OFF_B + SL_BSTAGE;

__device__ __forceinline__ int sl_tile_off(int m, int k) {   // canonical no-swizzle K-major, 64 columns
    return ((m >> 3) * 8 + (k >> 3)) * 64 + (m & 7) * 8 + (k & 7);
}
__device__ __forceinline__ float sl_pow2(int e) { return __int_as_float((127 + e) << 23); }   // e in [-126, 127]

// Moments -> B digit slices: one thread per (chunk, cluster, column n).  xh is the
// split layout [2R][C][q2]; out [nch][C][SL_S][SL_N][64] BF16 (canonical tiles),
// fexp [nch][C][SL_N] the column exponents (0 for an all-zero column).
__global__ void sliced_b_kernel(int R, int nch, int64_t C, const double* __restrict__ xh,
                                __nv_bfloat16* __restrict__ out, int* __restrict__ fexp) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nch * C * SL_N) return;
    const int n = (int)(idx % SL_N);
    const int64_t c = (idx / SL_N) % C;
    const int ch = (int)(idx / ((int64_t)SL_N * C));
    const int r = ch * SL_RQ + (n < SL_RQ ? n : n - SL_RQ);
    __nv_bfloat16* o = out + ((int64_t)ch * C + c) * SL_S * SL_N * SL_Q2;
    const double* src = r < R ? xh + ((int64_t)(2 * r + (n < SL_RQ ? 0 : 1)) * C + c) * SL_Q2 : nullptr;
    double mx = 0.0;
    if (src)
        for (int b = 0; b < SL_Q2; ++b) mx = fmax(mx, fabs(src[b]));
    int F = 0;
    if (mx > 0.0) frexp(mx, &F);               // |x| < 2^F
    fexp[idx] = F;
    const double sc = ldexp(1.0, 7 - F);
    for (int b = 0; b < SL_Q2; ++b) {
        double u = src ? src[b] * sc : 0.0;    // |u| < 128 before the first digit
        for (int s = 0; s < SL_S; ++s) {
            const double d = rint(u);
            o[s * SL_N * SL_Q2 + sl_tile_off(n, b)] = __float2bfloat16((float)d);
            u = (u - d) * 256.0;               // remainder in [-1/2, 1/2]: next digit in [-128, 128]
        }
    }
}

__device__ inline bool sl_wait(uint64_t* bar, unsigned parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(gsm(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ inline uint64_t sl_desc(unsigned addr) {   // LBO 128 B (K-adjacent core matrices), SBO 1024 B (8-row groups)
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46);
}
__device__ __forceinline__ void sl_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void sl_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(gsm(bar))
                 : "memory");
}

// One CTA per (target row sigma, chunk of 32 right-hand sides), 16 warps.
// Block i: K'_i is in the staging buffer Ks (generated while the tensor cores
// contracted block i - 1); once the MMAs of block i - 1 are done, the copies of
// B_i and of the points of block i + 1 are issued, the accumulators of block
// i - 1 are added into the row sums (kept in TMEM columns 384..511 as
// double-float hi, lo), K'_i is split into the SL_S A slices and, once B_i has
// landed, the 21 slice pairs are issued; then K'_{i+1} is generated into Ks.
// Thread (warp w, lane l) drains TMEM lane 32 (w % 4) + l and the 16 columns
// 16 (w / 4) .. + 15.
// pts [C][q2][2] float4 (hi, lo of x, y, z, k); xb [nch][C][SL_S][SL_N][64]
// BF16; fexp [nch][C][SL_N]; yh the split layout [2R][C][q2] doubles.
__global__ void __launch_bounds__(SL_THREADS, 1)
    helm_coupling_sliced_kernel(const int32_t* __restrict__ rows, const int64_t* __restrict__ fptr,
                                const int32_t* __restrict__ fsrc, const float4* __restrict__ pts,
                                const double* __restrict__ igeo, const float4* __restrict__ trig, GenConst gc, int R,
                                int64_t C, const __nv_bfloat16* __restrict__ xb, const int* __restrict__ fexp,
                                double* __restrict__ yh, long long wait_limit, int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + SL_OFF_BAR);   // fullY[0], fullY[1], fullB, done
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + SL_OFF_TSLOT);
    float* red = reinterpret_cast<float*>(smem + SL_OFF_RED);
    int* scs = reinterpret_cast<int*>(smem + SL_OFF_SC);               // [2][65]
    int* fst = reinterpret_cast<int*>(smem + SL_OFF_F);                // [2][64]
    float4* Xs = reinterpret_cast<float4*>(smem + SL_OFF_X);
    float4* Ys = reinterpret_cast<float4*>(smem + SL_OFF_Y);           // [2][2 q2]
    float4* Ks = reinterpret_cast<float4*>(smem + SL_OFF_K);           // [64][SL_KST]
    unsigned char* As = smem + SL_OFF_A;
    unsigned char* Bs = smem + SL_OFF_B;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int sigma = rows[blockIdx.x];
    const int chunk = blockIdx.y;
    const int64_t b0 = fptr[sigma];
    const int n = (int)(fptr[sigma + 1] - b0);
    const __nv_bfloat16* xc = xb + (int64_t)chunk * C * SL_S * SL_N * SL_Q2;
    const int* fc = fexp + (int64_t)chunk * C * SL_N;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const int cb = 16 * (warp >> 2);
    const int mrow = 32 * (warp & 3) + lane;

    auto issue_y = [&](int j) {   // points and column exponents of block j into stage j & 1 (thread 0)
        const int st = j & 1;
        const int64_t tau = fsrc[b0 + j];
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(gsm(&bars[st])),
                     "r"((unsigned)(2 * SL_Q2 * 16 + SL_N * 4))
                     : "memory");
        gen_bulk(Ys + st * 2 * SL_Q2, pts + tau * SL_Q2 * 2, 2 * SL_Q2 * 16, &bars[st]);
        gen_bulk(fst + st * SL_N, fc + tau * SL_N, SL_N * 4, &bars[st]);
    };
    auto issue_b = [&](int j) {   // B slices of block j (thread 0)
        const int64_t tau = fsrc[b0 + j];
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(gsm(&bars[2])),
                     "r"((unsigned)SL_BSTAGE)
                     : "memory");
        gen_bulk(Bs, xc + tau * SL_S * SL_N * SL_Q2, SL_BSTAGE, &bars[2]);
    };
    for (int k = tid; k < 2 * SL_Q2; k += SL_THREADS) Xs[k] = pts[(int64_t)sigma * SL_Q2 * 2 + k];
    if (tid == 0) {
        for (int k = 0; k < 4; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(gsm(&bars[k])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int j = 0; j < 2 && j < n; ++j) issue_y(j);
        if (n > 0) issue_b(0);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(gsm(tslot)), "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(SL_N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint32_t sum_hi = tmem + lane_base + (uint32_t)(SL_S * SL_N), sum_lo = sum_hi + SL_N;
    {   // row sums = 0
        uint32_t z[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) z[j] = 0u;
        for (int g8 = 0; g8 < 2; ++g8)
            for (int h = 0; h < 2; ++h)
                asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(
                                 (h ? sum_lo : sum_hi) + (uint32_t)(cb + 8 * g8)),
                             "r"(z[0]), "r"(z[1]), "r"(z[2]), "r"(z[3]), "r"(z[4]), "r"(z[5]), "r"(z[6]), "r"(z[7])
                             : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }

    // accumulators of the block whose scales are in scs[slot] -> row sums (TMEM)
    auto drain = [&](int slot) {
        const int E = scs[slot * 65 + 64];
        const float inv = 0.00390625f;   // 2^-8
#pragma unroll 1
        for (int g8 = 0; g8 < 2; ++g8) {
            const int c0 = cb + 8 * g8;
            uint32_t v[SL_S][8], hs[8], ls[8];
#pragma unroll
            for (int k = 0; k < SL_S; ++k)
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(v[k][0]), "=r"(v[k][1]), "=r"(v[k][2]), "=r"(v[k][3]), "=r"(v[k][4]),
                               "=r"(v[k][5]), "=r"(v[k][6]), "=r"(v[k][7])
                             : "r"(tmem + lane_base + (uint32_t)(k * SL_N + c0)));
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(hs[0]), "=r"(hs[1]), "=r"(hs[2]), "=r"(hs[3]), "=r"(hs[4]), "=r"(hs[5]),
                           "=r"(hs[6]), "=r"(hs[7])
                         : "r"(sum_hi + (uint32_t)c0));
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(ls[0]), "=r"(ls[1]), "=r"(ls[2]), "=r"(ls[3]), "=r"(ls[4]), "=r"(ls[5]),
                           "=r"(ls[6]), "=r"(ls[7])
                         : "r"(sum_lo + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                // sum_k 2^{-8k} D_k (exact integers below 2^23): FP32 for the
                // levels k >= 3 (their rounding stays below 2^-45 of the sum),
                // double-float from k = 2 down
                float T = fmaf(__uint_as_float(v[5][j]), inv, __uint_as_float(v[4][j]));
                T = fmaf(T, inv, __uint_as_float(v[3][j]));
                df acc = two_sum(__uint_as_float(v[2][j]), T * inv);
#pragma unroll
                for (int k = 1; k >= 0; --k) {
                    const df s2 = two_sum(__uint_as_float(v[k][j]), acc.h * inv);
                    acc = fast_two_sum(s2.h, s2.l + acc.l * inv);
                }
                // times 2^{E + F - 14}, in two exact power-of-two factors
                const int e = E + scs[slot * 65 + c0 + j] - 14;
                const int e1 = e / 2;
                const float f1 = sl_pow2(e1), f2 = sl_pow2(e - e1);
                const df sum = df_add({__uint_as_float(hs[j]), __uint_as_float(ls[j])},
                                      {acc.h * f1 * f2, acc.l * f1 * f2});
                hs[j] = __float_as_uint(sum.h);
                ls[j] = __float_as_uint(sum.l);
            }
            asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(
                             sum_hi + (uint32_t)c0),
                         "r"(hs[0]), "r"(hs[1]), "r"(hs[2]), "r"(hs[3]), "r"(hs[4]), "r"(hs[5]), "r"(hs[6]), "r"(hs[7])
                         : "memory");
            asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(
                             sum_lo + (uint32_t)c0),
                         "r"(ls[0]), "r"(ls[1]), "r"(ls[2]), "r"(ls[3]), "r"(ls[4]), "r"(ls[5]), "r"(ls[6]), "r"(ls[7])
                         : "memory");
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    };

    // K' of block j (points in stage j & 1) into Ks, its exponent E (|K'| < 2^E)
    // and the column exponents of its source into scs[j & 1]
    auto generate = [&](int j) {
        const int st = j & 1;
        float mx = 0.0f;
#pragma unroll 1
        for (int k = 0; k < 8; ++k) {
            const int v = tid + SL_THREADS * k;
            const int a = v >> 6, b = v & 63;
            df kr, ki;
            gen_entry(Xs[2 * a], Xs[2 * a + 1], Ys[st * 2 * SL_Q2 + 2 * b], Ys[st * 2 * SL_Q2 + 2 * b + 1], gc, trig,
                      kr, ki);
            Ks[a * SL_KST + b] = make_float4(kr.h, kr.l, ki.h, ki.l);
            mx = fmaxf(mx, fmaxf(fabsf(kr.h), fabsf(ki.h)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) red[warp] = mx;
        __syncthreads();
        float bm = red[0];
#pragma unroll
        for (int w = 1; w < SL_THREADS / 32; ++w) bm = fmaxf(bm, red[w]);
        int E = 0;
        if (bm > 0.0f) frexpf(bm, &E);
        if (tid < SL_N) scs[st * 65 + tid] = fst[st * SL_N + tid];
        if (tid == SL_N) scs[st * 65 + 64] = E;
        __syncthreads();   // the exponents are read by every thread
    };

    // the SL_S digits of K' (scaled by 2^{7 - E}) into the A slices: per thread two
    // groups of 8 consecutive columns of one row of [Re K'; Im K']
    auto emit = [&](int slot) {
        const float ps = sl_pow2(7 - scs[slot * 65 + 64]);
#pragma unroll 1
        for (int t2 = 0; t2 < 2; ++t2) {
            const int G = tid + SL_THREADS * t2;
            const int m = ((G >> 6) << 3) | (G & 7), b8 = (G >> 3) & 7;
            const int a = m & 63;
            const bool im = m >= SL_Q2;
            float yhi[8], ylo[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float4 kv = Ks[a * SL_KST + 8 * b8 + j];
                yhi[j] = (im ? kv.z : kv.x) * ps;
                ylo[j] = (im ? kv.w : kv.y) * ps;
            }
            unsigned char* dst = As + 2 * sl_tile_off(m, 8 * b8);
#pragma unroll 1
            for (int s = 0; s < SL_S; ++s) {
                uint32_t w[4];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float d = rintf(yhi[j]);
                    const df r = fast_two_sum(yhi[j] - d, ylo[j]);   // yhi - d is exact
                    yhi[j] = r.h * 256.0f;
                    ylo[j] = r.l * 256.0f;
                    const uint32_t bits = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(d));
                    if (j & 1)
                        w[j >> 1] |= bits << 16;
                    else
                        w[j >> 1] = bits;
                }
                *reinterpret_cast<uint4*>(dst + s * SL_ATILE) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    };

    // progress counters (uniform across the CTA) for the failure path
    int ycopies = n < 2 ? n : 2, ylanded = 0, bcopies = n > 0 ? 1 : 0, blanded = 0, issued = 0, done_waited = 0;
    bool failed = false;
    if (n > 0) {
        const bool ok = sl_wait(&bars[0], 0u, wait_limit);
        failed = __syncthreads_or(!ok);
        if (!failed) {
            ylanded = 1;
            generate(0);
        }
    }
    for (int i = 0; i < n && !failed; ++i) {
        if (i > 0) {
            // block i - 1 done: accumulators, A slices and B are free
            const bool ok = sl_wait(&bars[3], (unsigned)((i - 1) & 1), wait_limit);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            done_waited = issued;
            if (tid == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_b(i);
                if (i + 1 < n) issue_y(i + 1);
            }
            bcopies = i + 1;
            if (i + 1 < n) ycopies = i + 2;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            drain((i - 1) & 1);
        }
        emit(i & 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        const bool okb = sl_wait(&bars[2], (unsigned)(i & 1), wait_limit);   // B_i landed
        if (__syncthreads_or(!okb)) {
            failed = true;
            break;
        }
        blanded = i + 1;
        if (tid == 32) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int s = 0; s < SL_S; ++s)
                for (int t = 0; s + t < SL_S; ++t)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        sl_mma(tmem + (uint32_t)((s + t) * SL_N), sl_desc(gsm(As + s * SL_ATILE) + kk * 256),
                               sl_desc(gsm(Bs + t * SL_BTILE) + kk * 256), idesc, (s > 0 || kk > 0) ? 1u : 0u);
            sl_commit(&bars[3]);
        }
        issued = i + 1;
        if (i + 1 < n) {
            // K'_{i+1} while the tensor cores work on block i
            const bool ok = sl_wait(&bars[(i + 1) & 1], (unsigned)(((i + 1) >> 1) & 1), wait_limit);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            ylanded = i + 2;
            generate(i + 1);
        }
    }
    bool good = !failed;
    if (good && n > 0) {
        const bool ok = sl_wait(&bars[3], (unsigned)((n - 1) & 1), wait_limit);
        good = !__syncthreads_or(!ok);
        if (good) {
            done_waited = issued;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            drain((n - 1) & 1);
        }
    }
    if (!good) {
        // record, then let the copies and MMAs in flight finish (bounded) before the
        // accumulators are released
        if (tid == 0) {
            atomicOr(status, 1);
            for (int j = ylanded; j < ycopies; ++j) sl_wait(&bars[j & 1], (unsigned)((j >> 1) & 1), 1LL << 24);
            if (bcopies > blanded) sl_wait(&bars[2], (unsigned)((bcopies - 1) & 1), 1LL << 24);
            if (issued > done_waited) sl_wait(&bars[3], (unsigned)((issued - 1) & 1), 1LL << 24);
        }
    } else {
        // row sums TMEM -> shared memory (the A slices are free), real form, k_a / (4 pi)
        float2* S = reinterpret_cast<float2*>(As);   // [128][SL_N]
#pragma unroll 1
        for (int g8 = 0; g8 < 2; ++g8) {
            const int c0 = cb + 8 * g8;
            uint32_t hs[8], ls[8];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(hs[0]), "=r"(hs[1]), "=r"(hs[2]), "=r"(hs[3]), "=r"(hs[4]), "=r"(hs[5]),
                           "=r"(hs[6]), "=r"(hs[7])
                         : "r"(sum_hi + (uint32_t)c0));
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(ls[0]), "=r"(ls[1]), "=r"(ls[2]), "=r"(ls[3]), "=r"(ls[4]), "=r"(ls[5]),
                           "=r"(ls[6]), "=r"(ls[7])
                         : "r"(sum_lo + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 8; ++j)
                S[mrow * SL_N + c0 + j] = make_float2(__uint_as_float(hs[j]), __uint_as_float(ls[j]));
        }
        __syncthreads();
        for (int e = tid; e < SL_Q2 * SL_RQ; e += SL_THREADS) {
            const int a = e / SL_RQ, r = e % SL_RQ;
            const int rg = chunk * SL_RQ + r;
            if (rg >= R) continue;
            const float2 p = S[a * SL_N + r], q = S[(SL_Q2 + a) * SL_N + SL_RQ + r];
            const float2 u = S[a * SL_N + SL_RQ + r], v = S[(SL_Q2 + a) * SL_N + r];
            const double ka = igeo[4 * ((int64_t)sigma * SL_Q2 + a) + 3] / (4.0 * IBEM_PI);
            const double re = (((double)p.x + (double)p.y) - ((double)q.x + (double)q.y)) * ka;
            const double im = (((double)u.x + (double)u.y) + ((double)v.x + (double)v.y)) * ka;
            yh[((int64_t)(2 * rg) * C + sigma) * SL_Q2 + a] = re;
            yh[((int64_t)(2 * rg + 1) * C + sigma) * SL_Q2 + a] = im;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

float round_bits(long double v, int bits) {
    if (v == 0.0L) return 0.0f;
    int ex;
    std::frexp((double)v, &ex);
    const long double scale = std::ldexp(1.0L, bits - ex);
    return (float)(std::nearbyint(v * scale) / scale);
}

}  // namespace

// q <= 8 (a generated block fits in shared memory) and a phase kappa r below
// 90 on every far block (n < 2^15 keeps the products n c_1..3 exact)
bool gen_supported(const ibem_handle* h) {
    return h->helm && h->P.q > 0 && h->P.q2 <= 64 && h->P.prm.kappa * h->far_diam < 90.0;
}

// point table and e^{i j c} table of the double-float generation (once per handle)
static cudaError_t ensure_gen_tables(ibem_handle* h) {
    Plan& P = h->P;
    cudaStream_t st = h->stream;
    cudaError_t e;
    const int q2 = P.q2;
    const int T = 256;
    if (!h->d_gen_pts) {
        if ((e = cudaMalloc(&h->d_gen_pts, (size_t)P.C * q2 * 2 * sizeof(float4)))) return e;
        gen_points_kernel<<<nblk(P.C * q2, T), T, 0, st>>>(P.C * q2, h->d_igeo, h->d_gen_pts);
        // e^{i j c}, c = 2 pi / GEN_TABLE, as double-float pairs (host, extended precision)
        std::vector<float4> tab(GEN_TABLE);
        const long double two_pi = 6.283185307179586476925286766559005768L;
        for (int j = 0; j < GEN_TABLE; ++j) {
            const long double a = two_pi * j / GEN_TABLE;
            const long double c = std::cos(a), s = std::sin(a);
            const float ch = (float)c, sh = (float)s;
            tab[j] = make_float4(ch, (float)(c - ch), sh, (float)(s - sh));
        }
        if ((e = cudaMalloc(&h->d_gen_trig, GEN_TABLE * sizeof(float4)))) return e;
        if ((e = cudaMemcpyAsync(h->d_gen_trig, tab.data(), GEN_TABLE * sizeof(float4), cudaMemcpyHostToDevice, st)))
            return e;
        if ((e = cudaStreamSynchronize(st))) return e;
    }
    return cudaSuccess;
}

// kappa as double-float, 1 / c and the four-part split of c = 2 pi / GEN_TABLE
static GenConst gen_constants(const Plan& P) {
    GenConst g;
    g.kh = (float)P.prm.kappa;
    g.kl = (float)(P.prm.kappa - (double)g.kh);
    const long double c = 6.283185307179586476925286766559005768L / GEN_TABLE;
    g.inv_c = (float)(1.0L / c);
    g.c1 = round_bits(c, 9);
    g.c2 = round_bits(c - g.c1, 9);
    g.c3 = round_bits(c - g.c1 - g.c2, 9);
    g.c4 = (float)(c - g.c1 - g.c2 - g.c3);
    return g;
}

cudaError_t launch_coupling_gen(ibem_handle* h, int R) {
    Plan& P = h->P;
    cudaStream_t st = h->stream;
    cudaError_t e;
    const int q2 = P.q2;
    const int T = 256;
    if ((e = ensure_gen_tables(h))) return e;
    const int RC = R <= 16 ? 16 : (R <= 32 ? 32 : 64);
    const int nch = (R + RC - 1) / RC;
    const size_t xbytes = (size_t)nch * P.C * q2 * RC * sizeof(float4);
    if (xbytes > h->gen_x_bytes) {
        cudaFree(h->d_gen_x);
        h->d_gen_x = nullptr;
        h->gen_x_bytes = 0;
        if ((e = cudaMalloc(&h->d_gen_x, xbytes))) return e;
        h->gen_x_bytes = xbytes;
    }
    gen_split_kernel<<<nblk((int64_t)nch * P.C * q2 * RC, T), T, 0, st>>>(R, RC, nch, P.C, q2, h->d_xh, h->d_gen_x);
    const GenConst g = gen_constants(P);
    const size_t sm = gen_smem_bytes(q2, RC);
    const unsigned nrows = (unsigned)h->far_rows.size();
    dim3 grid(nrows, nch);
#define IBEM_GEN_LAUNCH(RC_)                                                                                      \
    if ((e = cudaFuncSetAttribute(helm_coupling_gen_kernel<RC_>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                  (int)sm)))                                                                    \
        return e;                                                                                               \
    helm_coupling_gen_kernel<RC_><<<grid, GEN_THREADS, sm, st>>>(                                               \
        h->d_far_rows, h->d_far_ptr, h->d_far_src, h->d_gen_pts, h->d_igeo, h->d_gen_trig, g, q2, R, P.C,       \
        h->d_gen_x, h->d_yh, h->wait_limit, h->d_status);
    if (RC == 16) {
        IBEM_GEN_LAUNCH(16)
    } else if (RC == 32) {
        IBEM_GEN_LAUNCH(32)
    } else {
        IBEM_GEN_LAUNCH(64)
    }
#undef IBEM_GEN_LAUNCH
    h->launches += 2;
    return cudaGetLastError();
}

bool sliced_supported(const ibem_handle* h) {
    return h->helm && h->P.q2 == SL_Q2 && h->P.prm.kappa * h->far_diam < 90.0;
}

// FP64-accurate coupling by digit slices on the tensor cores (q = 8): the moments
// are sliced once per application, then one CTA per (target row, chunk of 32
// right-hand sides) generates, slices and contracts every far block of its row.
cudaError_t launch_coupling_sliced(ibem_handle* h, int R) {
    Plan& P = h->P;
    cudaStream_t st = h->stream;
    cudaError_t e;
    const int T = 256;
    if ((e = ensure_gen_tables(h))) return e;
    const int nch = (R + SL_RQ - 1) / SL_RQ;
    const size_t xbytes = (size_t)nch * P.C * SL_BSTAGE, fbytes = (size_t)nch * P.C * SL_N * sizeof(int);
    if (xbytes + fbytes > h->sl_bytes) {
        cudaFree(h->d_sl);
        h->d_sl = nullptr;
        h->sl_bytes = 0;
        if ((e = cudaMalloc(&h->d_sl, xbytes + fbytes))) return e;
        h->sl_bytes = xbytes + fbytes;
    }
    __nv_bfloat16* xb = reinterpret_cast<__nv_bfloat16*>(h->d_sl);
    int* fexp = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(h->d_sl) + xbytes);
    sliced_b_kernel<<<nblk((int64_t)nch * P.C * SL_N, T), T, 0, st>>>(R, nch, P.C, h->d_xh, xb, fexp);
    const GenConst g = gen_constants(P);
    if ((e = cudaFuncSetAttribute(helm_coupling_sliced_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SL_SMEM)))
        return e;
    const unsigned nrows = (unsigned)h->far_rows.size();
    helm_coupling_sliced_kernel<<<dim3(nrows, (unsigned)nch), SL_THREADS, SL_SMEM, st>>>(
        h->d_far_rows, h->d_far_ptr, h->d_far_src, h->d_gen_pts, h->d_igeo, h->d_gen_trig, g, R, P.C, xb, fexp,
        h->d_yh, h->wait_limit, h->d_status);
    h->launches += 2;
    return cudaGetLastError();
}

}  // namespace ibem
