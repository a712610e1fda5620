// Learned right preconditioner (no counterpart in the paper, which uses Jacobi
// preconditioning, Sec. 4 item 3): a small convolutional network on the
// B-spline coefficient grid of each patch, used as a correction of block-Jacobi
// inside flexible GMRES.
//
// A complex vector of S_{p,m} is, patch by patch, an image with 2 channels
// (real, imaginary part) of n1 x n1 pixels (pixel (jv, ju) = dof (patch, ju, jv)).
// Network: four 3 x 3 convolutions (2 -> C -> C -> C -> 2 channels, zero
// padding), ReLU after the first three; parameters flat, layer by layer,
// W[cout][cin][3][3] then bias[cout], kept in FP32 with the Adam moments.
// BF16 mode stores activations in BF16 and rounds the weights to BF16 where they
// are used, with FP32 accumulation; FP32 mode keeps everything in FP32.
//
// Preconditioner: s = B^-1 v (block-Jacobi), sigma = |s| / sqrt(2N),
// z = s + sigma * net(s / sigma), the network in BF16.
//
// Kernels: inference in BF16 (the preconditioner, ibem_cnn_forward) runs all
// four layers on the tensor cores (tcgen05 implicit GEMM, conv_tc_kernel).
// Training and the FP32 mode use one tiled direct convolution (16 x 16 output
// pixels of one image and 16 output channels per CTA, input halo tile and
// weights staged in shared memory, FP32 FMA) for the forward pass and, with
// flipped transposed weights and the ReLU mask fused, the input gradient; the
// weight gradient is a tiled reduction over pixels into per-CTA partial sums
// that a second kernel adds in a fixed order, so training is deterministic.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>

#include "ibem_internal.cuh"

struct ibem_cnn {
    int C = 32;                  // hidden channels
    int L = 4;                   // layers
    std::vector<int> cin, cout;  // per layer
    std::vector<size_t> woff, boff;
    size_t nparam = 0;
    int device = 0;
    float* d_param = nullptr;    // weights and biases, FP32
    float* d_grad = nullptr;
    float* d_m = nullptr;        // Adam moments
    float* d_v = nullptr;
    float* d_wt = nullptr;       // flipped transposed weights of one layer (backward)
    int64_t step = 0;
    void* d_act = nullptr;       // activations of the last forward pass: L + 1 slots
    size_t act_slot = 0;         // elements per slot
    size_t act_bytes = 0;
    float* d_gbuf = nullptr;     // two gradient buffers, act_slot floats each
    size_t gbuf_floats = 0;
    float* d_part = nullptr;     // weight-gradient partial sums
    size_t part_floats = 0;
    float* d_img = nullptr;      // preconditioner / training batch images
    size_t img_floats = 0;
    void* d_items = nullptr;     // training minibatch items of one epoch
    size_t items_bytes = 0;
    void* d_opvec = nullptr;     // residual-norm objective: vectors
    size_t opvec_bytes = 0;
    void* d_opimg = nullptr;     // residual-norm objective: images
    size_t opimg_bytes = 0;
    void* d_wtc = nullptr;       // BF16 tensor-core weight tiles of the four layers
    size_t wtc_bytes = 0;
    int* d_status = nullptr;     // device-side wait status of the tensor-core layers
    double* d_red = nullptr;     // [0] loss, [1] |s|^2, [2] loss sum of an epoch
    int coarse = 1;              // coarsening factor f of the preconditioner's images (1: the fine grid)
    float* d_cimg = nullptr;     // coarse images of the preconditioner
    size_t cimg_floats = 0;
    cudaStream_t stream = nullptr;
    int64_t launches = 0;
};

namespace ibem {

namespace {

constexpr int TS = 16;        // output tile side
constexpr int CIB = 8;        // input channels per shared-memory stage
constexpr int WG_ITEMS = 256; // CTAs along the pixel axis of the weight gradient

inline unsigned cblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

__device__ inline float ld_act(const float* p, int64_t i) { return p[i]; }
__device__ inline float ld_act(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }
__device__ inline void st_act(float* p, int64_t i, float v) { p[i] = v; }
__device__ inline void st_act(__nv_bfloat16* p, int64_t i, float v) { p[i] = __float2bfloat16(v); }
__device__ inline float wq(float w, int bf) { return bf ? __bfloat162float(__float2bfloat16(w)) : w; }

// out[b][co][y][x] = bias[co] + sum_ci sum_k w[co][ci][k] in[b][ci][y + dy - 1][x + dx - 1]
// (k = 3 dy + dx), then ReLU if relu, then zeroed where mask[b][co][y][x] <= 0
// if mask is given.  Grid: (tiles of the image, ceil(Cout / COB), B).
template <typename TI, typename TO, typename TM, int COB>
__global__ void __launch_bounds__(256) conv_tile_kernel(const TI* __restrict__ in, int Cin, int H, int W,
                                                        const float* __restrict__ w,
                                                        const float* __restrict__ bias, int Cout, int relu, int bf,
                                                        const TM* __restrict__ mask, TO* __restrict__ out) {
    __shared__ float s_in[CIB][TS + 2][TS + 2];
    __shared__ __align__(16) float s_w[CIB][9][COB];
    const int tiles_x = (W + TS - 1) / TS;
    const int ty0 = (blockIdx.x / tiles_x) * TS, tx0 = (blockIdx.x % tiles_x) * TS;
    const int co0 = blockIdx.y * COB;
    const int64_t b = blockIdx.z;
    const int t = threadIdx.x, py = t / TS, px = t % TS;
    const int y = ty0 + py, x = tx0 + px;
    const int64_t HW = (int64_t)H * W;
    float acc[COB];
#pragma unroll
    for (int c = 0; c < COB; ++c) acc[c] = (bias && co0 + c < Cout) ? bias[co0 + c] : 0.0f;
    for (int ci0 = 0; ci0 < Cin; ci0 += CIB) {
        for (int i = t; i < CIB * (TS + 2) * (TS + 2); i += 256) {
            const int c = i / ((TS + 2) * (TS + 2)), r = i % ((TS + 2) * (TS + 2));
            const int yy = ty0 - 1 + r / (TS + 2), xx = tx0 - 1 + r % (TS + 2);
            float v = 0.0f;
            if (ci0 + c < Cin && yy >= 0 && yy < H && xx >= 0 && xx < W)
                v = ld_act(in, (b * Cin + ci0 + c) * HW + (int64_t)yy * W + xx);
            s_in[c][r / (TS + 2)][r % (TS + 2)] = v;
        }
        for (int i = t; i < CIB * 9 * COB; i += 256) {
            const int co = i % COB, k = (i / COB) % 9, c = i / (9 * COB);
            float v = 0.0f;
            if (ci0 + c < Cin && co0 + co < Cout) v = wq(w[((int64_t)(co0 + co) * Cin + ci0 + c) * 9 + k], bf);
            s_w[c][k][co] = v;
        }
        __syncthreads();
        const int cmax = min(CIB, Cin - ci0);
        for (int c = 0; c < cmax; ++c) {
            float v[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) v[k] = s_in[c][py + k / 3][px + k % 3];
#pragma unroll
            for (int k = 0; k < 9; ++k)
#pragma unroll
                for (int co = 0; co < COB; ++co) acc[co] = fmaf(s_w[c][k][co], v[k], acc[co]);
        }
        __syncthreads();
    }
    if (y >= H || x >= W) return;
#pragma unroll
    for (int co = 0; co < COB; ++co) {
        if (co0 + co >= Cout) break;
        float r = acc[co];
        if (relu && r < 0.0f) r = 0.0f;
        const int64_t o = (b * Cout + co0 + co) * HW + (int64_t)y * W + x;
        if (mask && !(ld_act(mask, o) > 0.0f)) r = 0.0f;
        st_act(out, o, r);
    }
}

// ---- inference layers on the tensor cores -----------------------------------------
// Implicit GEMM: D[m][co] = sum over taps (dy, dx) and input channels of
// A_tap[m][ci] W_tap[co][ci], with m an output position in padded-pitch order
// o = y * P + x (P = W + 2; columns x >= W are computed and discarded).  The
// input positions of tap (dy, dx) are o + dy * P + dx in the zero-padded
// image, so one shared-memory band of padded rows serves all nine taps: tap
// (dy, dx) is the same band started dy * P + dx rows later.  Band layout
// (tcgen05 canonical K-major, no swizzle): channel group g (8 channels, 16
// bytes) of band row r at (g * NBP + r) * 16 bytes, so rows are contiguous
// (core-matrix stride along M = 128 B) and the channel groups are NBP * 16 B
// apart (stride along K).  Weights per tap: core (co / 8, ci / 8) at
// ((co / 8) * KG + ci / 8) * 128 B.  A tile is TC_MB blocks of 128 consecutive
// positions sharing one band of TC_MB * 128 + 2P + 2 rows (copied with cp.async,
// zero-filled outside the image); each block accumulates in its own 32 TMEM
// columns (tcgen05.mma kind::f16, M = 128, N = NP, K = 16, BF16 operands, FP32
// accumulation), and all MMAs of a tile are committed once.  Epilogue: bias,
// optional ReLU, BF16 store.
//   CGI: channel groups of an input pixel (1: the 2-channel input padded to 8
//        channels, 4: 32 channels); the band holds KG = max(CGI, 2) groups
//        (the second group of a 1-group input is zero, and so are its weights).
//   NP:  MMA width (32, or 16 for the 2-channel output layer); NOUT channels kept.
//   OUT_PLANAR: output [B][NOUT][H][W] (last layer) instead of pixel-major.
constexpr int TC_M = 128;
constexpr int TC_MB = 4;

__device__ inline unsigned cnn_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ inline uint64_t cnn_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ inline bool cnn_wait(uint64_t* bar, unsigned parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(cnn_smem(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// w [Cout][Cin][9] FP32 -> BF16 canonical tiles [9][NP / 8][KG][8][8] (zero padded)
__global__ void tc_weights_kernel(const float* __restrict__ w, int Cin, int Cout, int NP, int KG,
                                  __nv_bfloat16* __restrict__ wt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int CI = 8 * KG;
    if (i >= NP * CI * 9) return;
    const int k = i % 9, ci = (i / 9) % CI, co = i / (9 * CI);
    const float v = (co < Cout && ci < Cin) ? w[((int64_t)co * Cin + ci) * 9 + k] : 0.0f;
    wt[(k * (NP / 8) * KG + (co >> 3) * KG + (ci >> 3)) * 64 + (co & 7) * 8 + (ci & 7)] = __float2bfloat16(v);
}

// FP32 planar [B][2][H][W] -> BF16 pixel-major [B][H][W][8] (channels 2..7 zero)
__global__ void pack8_kernel(int64_t npx, int64_t HW, const float* __restrict__ in, __nv_bfloat16* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npx) return;
    const int64_t b = i / HW, pix = i % HW;
    __nv_bfloat162 v = __floats2bfloat162_rn(in[(b * 2) * HW + pix], in[(b * 2 + 1) * HW + pix]);
    *reinterpret_cast<uint4*>(out + i * 8) = make_uint4(*reinterpret_cast<uint32_t*>(&v), 0u, 0u, 0u);
}

// Persistent CTAs of 128 threads (one output position per thread and block).
template <int CGI, int NP, int NOUT, bool OUT_PLANAR>
__global__ void __launch_bounds__(128) conv_tc_kernel(const __nv_bfloat16* __restrict__ in, int B, int H, int W,
                                                      const __nv_bfloat16* __restrict__ wt,
                                                      const float* __restrict__ bias, int relu, int nbp,
                                                      __nv_bfloat16* __restrict__ out, long long wait_limit,
                                                      int* __restrict__ status) {
    constexpr int KG = CGI < 2 ? 2 : CGI;
    constexpr int WBYTES = 9 * (NP / 8) * KG * 128;
    constexpr int TILE = TC_M * TC_MB;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* wsm = smem;
    unsigned char* band = smem + WBYTES;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(band + KG * nbp * 16);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int P = W + 2;
    const int64_t tiles_img = ((int64_t)H * P + TILE - 1) / TILE;
    const int64_t ntiles = (int64_t)B * tiles_img;
    const int nb = TILE + 2 * P + 2;
    for (int i = t; i < WBYTES / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(wsm)[i] = reinterpret_cast<const uint4*>(wt)[i];
    if (CGI < KG)   // zero channel group of a 1-group input
        for (int r = t; r < nbp; r += blockDim.x)
            *reinterpret_cast<uint4*>(band + ((size_t)1 * nbp + r) * 16) = make_uint4(0u, 0u, 0u, 0u);
    float bv[NOUT];
#pragma unroll
    for (int c = 0; c < NOUT; ++c) bv[c] = bias[c];
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cnn_smem(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(cnn_smem(tslot)),
                     "r"(32 * TC_MB)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NP >> 3) << 17) |
                           ((uint32_t)(TC_M >> 4) << 24);
    // descriptors of offset 0; an operand starting k * 16 bytes later is desc + k
    // (the start-address field counts 16-byte units; all addresses < 256 KB)
    const uint64_t adesc0 = cnn_desc(cnn_smem(band), nbp * 16, 128);
    const uint64_t bdesc0 = cnn_desc(cnn_smem(wsm), 128, KG * 128);
    int it = 0;
    bool failed = false;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int64_t b = tile / tiles_img;
        const int o0 = (int)((tile % tiles_img) * TILE);
        // band of padded rows o0 .. o0 + nb - 1: all 16-byte copies in flight at
        // once (cp.async), zero-filled outside the image (source size 0)
        for (int idx = t; idx < nb * CGI; idx += blockDim.x) {
            const int r = idx / CGI, g = idx % CGI;
            const int i = o0 + r;
            const int py = i / P, px = i - py * P;
            const bool inside = py >= 1 && py <= H && px >= 1 && px <= W;
            const __nv_bfloat16* s = inside ? in + ((b * H + (py - 1)) * W + (px - 1)) * (8 * CGI) + g * 8 : in;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                             cnn_smem(band + ((size_t)g * nbp + r) * 16)),
                         "l"(s), "r"(inside ? 16u : 0u)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (t == 0) {
#pragma unroll 1
            for (int mb = 0; mb < TC_MB; ++mb)
#pragma unroll 1
                for (int tap = 0; tap < 9; ++tap) {
                    const int roff = mb * TC_M + (tap / 3) * P + (tap % 3);
                    for (int s = 0; s < KG / 2; ++s) {
                        const uint64_t ad = adesc0 + (uint64_t)(2 * s * nbp + roff);
                        const uint64_t bd = bdesc0 + (uint64_t)(tap * (NP / 8) * KG * 8 + 2 * s * 8);
                        const uint32_t acc = (tap > 0 || s > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem + 32u * mb),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             cnn_smem(mbar))
                         : "memory");
        }
        const bool ok = cnn_wait(mbar, (unsigned)(it & 1), wait_limit);
        if (__syncthreads_or(!ok)) {
            // the MMAs may still run: wait for them (bounded) before the band is released
            cnn_wait(mbar, (unsigned)(it & 1), 1LL << 24);
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
        for (int mb = 0; mb < TC_MB; ++mb) {
            const int o = o0 + mb * TC_M + 32 * warp + lane;
            const int y = o / P, x = o - y * P;
            uint32_t v[NP];
#pragma unroll
            for (int c0 = 0; c0 < NP; c0 += 16) {
                const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * mb + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[c0 + 0]), "=r"(v[c0 + 1]), "=r"(v[c0 + 2]), "=r"(v[c0 + 3]), "=r"(v[c0 + 4]),
                      "=r"(v[c0 + 5]), "=r"(v[c0 + 6]), "=r"(v[c0 + 7]), "=r"(v[c0 + 8]), "=r"(v[c0 + 9]),
                      "=r"(v[c0 + 10]), "=r"(v[c0 + 11]), "=r"(v[c0 + 12]), "=r"(v[c0 + 13]), "=r"(v[c0 + 14]),
                      "=r"(v[c0 + 15])
                    : "r"(taddr));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (y < H && x < W) {
                if constexpr (OUT_PLANAR) {
#pragma unroll
                    for (int co = 0; co < NOUT; ++co) {
                        float f = __uint_as_float(v[co]) + bv[co];
                        if (relu) f = fmaxf(f, 0.0f);
                        out[((b * NOUT + co) * H + y) * (int64_t)W + x] = __float2bfloat16(f);
                    }
                } else {
                    uint4* dst = reinterpret_cast<uint4*>(out + ((b * H + y) * W + x) * NOUT);
#pragma unroll
                    for (int q4 = 0; q4 < NOUT / 8; ++q4) {
                        uint32_t pk[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            float f0 = __uint_as_float(v[q4 * 8 + 2 * j]) + bv[q4 * 8 + 2 * j];
                            float f1 = __uint_as_float(v[q4 * 8 + 2 * j + 1]) + bv[q4 * 8 + 2 * j + 1];
                            if (relu) {
                                f0 = fmaxf(f0, 0.0f);
                                f1 = fmaxf(f1, 0.0f);
                            }
                            __nv_bfloat162 h2 = __floats2bfloat162_rn(f0, f1);
                            pk[j] = *reinterpret_cast<uint32_t*>(&h2);
                        }
                        dst[q4] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    }
                }
            }
        }
        // the next tile rewrites the band and the accumulators
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (failed && t == 0) atomicOr(status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32 * TC_MB)
                     : "memory");
}

// wt[ci][co][k] = w[co][ci][8 - k] (rounded to BF16 in BF16 mode): the kernel of
// the input gradient, which is a convolution of the output gradient with the
// flipped, channel-transposed weights.
__global__ void flip_weights_kernel(const float* __restrict__ w, int Cin, int Cout, int bf, float* __restrict__ wt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Cin * Cout * 9) return;
    const int k = i % 9, co = (i / 9) % Cout, ci = i / (9 * Cout);
    wt[i] = wq(w[((int64_t)co * Cin + ci) * 9 + (8 - k)], bf);
}

// Partial weight gradients: CTA (x, y) sums, over its range of (image, tile)
// items, g[b][co][pix] * in[b][ci][pix + tap] for co < Cout (<= 32), the 8
// input channels of chunk y and the 9 taps; thread = (ci within chunk, co).
template <typename T>
__global__ void __launch_bounds__(256) conv_wgrad_kernel(const float* __restrict__ g, const T* __restrict__ in, int B,
                                                         int Cin, int H, int W, int Cout, int items_per_cta,
                                                         float* __restrict__ part) {
    __shared__ float s_g[32][TS * TS + 1];
    __shared__ float s_in[CIB][TS + 2][TS + 2];
    const int tiles_x = (W + TS - 1) / TS, tiles = tiles_x * ((H + TS - 1) / TS);
    const int64_t HW = (int64_t)H * W;
    const int t = threadIdx.x, co = t % 32, c = t / 32;
    const int ci0 = blockIdx.y * CIB;
    const int64_t it0 = (int64_t)blockIdx.x * items_per_cta;
    const int64_t it1 = min((int64_t)B * tiles, it0 + items_per_cta);
    float acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
    for (int64_t item = it0; item < it1; ++item) {
        const int64_t b = item / tiles;
        const int tile = (int)(item % tiles);
        const int ty0 = (tile / tiles_x) * TS, tx0 = (tile % tiles_x) * TS;
        for (int i = t; i < Cout * TS * TS; i += 256) {
            const int o = i / (TS * TS), pix = i % (TS * TS);
            const int yy = ty0 + pix / TS, xx = tx0 + pix % TS;
            s_g[o][pix] = (yy < H && xx < W) ? g[(b * Cout + o) * HW + (int64_t)yy * W + xx] : 0.0f;
        }
        for (int i = t; i < CIB * (TS + 2) * (TS + 2); i += 256) {
            const int cc = i / ((TS + 2) * (TS + 2)), r = i % ((TS + 2) * (TS + 2));
            const int yy = ty0 - 1 + r / (TS + 2), xx = tx0 - 1 + r % (TS + 2);
            float v = 0.0f;
            if (ci0 + cc < Cin && yy >= 0 && yy < H && xx >= 0 && xx < W)
                v = ld_act(in, (b * Cin + ci0 + cc) * HW + (int64_t)yy * W + xx);
            s_in[cc][r / (TS + 2)][r % (TS + 2)] = v;
        }
        __syncthreads();
        if (co < Cout && ci0 + c < Cin) {
            for (int py = 0; py < TS; ++py) {
                // 3 x 3 window slid along the row: three new values per pixel
                float w0[3], w1[3];
#pragma unroll
                for (int dy = 0; dy < 3; ++dy) {
                    w0[dy] = s_in[c][py + dy][0];
                    w1[dy] = s_in[c][py + dy][1];
                }
                for (int px = 0; px < TS; ++px) {
                    float w2[3];
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy) w2[dy] = s_in[c][py + dy][px + 2];
                    const float gv = s_g[co][py * TS + px];
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy) {
                        acc[dy * 3 + 0] = fmaf(gv, w0[dy], acc[dy * 3 + 0]);
                        acc[dy * 3 + 1] = fmaf(gv, w1[dy], acc[dy * 3 + 1]);
                        acc[dy * 3 + 2] = fmaf(gv, w2[dy], acc[dy * 3 + 2]);
                        w0[dy] = w1[dy];
                        w1[dy] = w2[dy];
                    }
                }
            }
        }
        __syncthreads();
    }
    if (co < Cout && ci0 + c < Cin) {
        float* dst = part + (int64_t)blockIdx.x * Cout * Cin * 9 + ((int64_t)co * Cin + ci0 + c) * 9;
#pragma unroll
        for (int k = 0; k < 9; ++k) dst[k] = acc[k];
    }
}

// gw[i] = sum over rows r (in order) of part[r][i]
__global__ void sum_rows_kernel(const float* __restrict__ part, int rows, int n, float* __restrict__ gw) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.0f;
    for (int r = 0; r < rows; ++r) s += part[(int64_t)r * n + i];
    gw[i] = s;
}

// gb[co] = sum over b and pixels of g[b][co][.]; one CTA per channel
__global__ void bias_grad_kernel(const float* __restrict__ g, int B, int Cout, int64_t HW, float* __restrict__ gb) {
    __shared__ float red[256];
    const int co = blockIdx.x;
    float s = 0.0f;
    for (int64_t i = threadIdx.x; i < (int64_t)B * HW; i += blockDim.x) s += g[((i / HW) * Cout + co) * HW + i % HW];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) gb[co] = red[0];
}

// g = (out - target) / B; loss[0] = 1/(2B) sum (out - target)^2; loss[2] += B * loss[0]
template <typename T>
__global__ void loss_kernel(int64_t n, int B, const T* __restrict__ out, const float* __restrict__ target,
                            float* __restrict__ g, double* __restrict__ loss) {
    __shared__ double red[1024];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const float d = ld_act(out, i) - target[i];
        g[i] = d / B;
        acc += (double)d * d;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        loss[0] = red[0] / (2.0 * B);
        loss[2] += red[0] / 2.0;
    }
}

__global__ void adam_kernel(size_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

template <typename T>
__global__ void f32_to_act_kernel(int64_t n, const float* __restrict__ in, T* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) st_act(out, i, in[i]);
}

template <typename T>
__global__ void act_to_f32_kernel(int64_t n, const T* __restrict__ in, float* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ld_act(in, i);
}

// One training image of a minibatch: source index, symmetry of the square and
// phase rotation (cos, sin) applied to input and target alike.
struct TrainItem {
    int src;
    int dihedral;
    float c, s;
};

// dihedral d: optionally transpose (bit 2), then mirror rows (bit 0) and
// columns (bit 1); out[j][ch][y][x] = rotate(in[src][.][sy][sx])
__global__ void gather_kernel(int nb, int H, int W, const TrainItem* __restrict__ items, const float* __restrict__ in,
                              const float* __restrict__ tgt, float* __restrict__ bin, float* __restrict__ btgt) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t HW = (int64_t)H * W;
    if (idx >= (int64_t)nb * HW) return;
    const int j = (int)(idx / HW);
    const int y = (int)((idx % HW) / W), x = (int)(idx % W);
    const TrainItem it = items[j];
    int a = y, bcol = x;
    if (it.dihedral & 4) { a = x; bcol = y; }
    if (it.dihedral & 1) a = H - 1 - a;
    if (it.dihedral & 2) bcol = W - 1 - bcol;
    const int64_t s0 = ((int64_t)it.src * 2) * HW + (int64_t)a * W + bcol;
    const int64_t d0 = ((int64_t)j * 2) * HW + (int64_t)y * W + x;
    float re = in[s0], im = in[s0 + HW];
    bin[d0] = it.c * re - it.s * im;
    bin[d0 + HW] = it.s * re + it.c * im;
    re = tgt[s0];
    im = tgt[s0 + HW];
    btgt[d0] = it.c * re - it.s * im;
    btgt[d0 + HW] = it.s * re + it.c * im;
}

// Coarse grid of the preconditioner (factor f): the mean over blocks of f x f
// pixels (ragged blocks at the far edge average the pixels they hold), and the
// block sums (the adjoint of the piecewise-constant prolongation, for the
// gradient).  Images [n_ch][n1][n1] -> [n_ch][nc][nc], nc = ceil(n1 / f).
__global__ void restrict_images_kernel(int64_t n_ch, int n1, int f, int nc, const float* __restrict__ in,
                                       float* __restrict__ out, int mean) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_ch * nc * nc) return;
    const int X = (int)(idx % nc), Y = (int)((idx / nc) % nc);
    const int64_t ch = idx / ((int64_t)nc * nc);
    const float* src = in + ch * n1 * n1;
    const int y1 = min(n1, (Y + 1) * f), x1 = min(n1, (X + 1) * f);
    float acc = 0.0f;
    for (int y = Y * f; y < y1; ++y)
        for (int x = X * f; x < x1; ++x) acc += src[(int64_t)y * n1 + x];
    out[idx] = mean ? acc / (float)((y1 - Y * f) * (x1 - X * f)) : acc;
}

// Preconditioner glue.  img[patch][2][n1][n1] = s / sigma with
// sigma^2 = |s|^2 / (2N) (zero image if s = 0).
__global__ void pack_images_kernel(int64_t N, int n1, const double* __restrict__ s, const double* __restrict__ ss,
                                   float* __restrict__ img) {
    int64_t dof = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (dof >= N) return;
    const int64_t per = (int64_t)n1 * n1;
    const int64_t patch = dof / per, pix = dof % per;
    const double inv = ss[0] > 0.0 ? 1.0 / sqrt(ss[0] / (2.0 * N)) : 0.0;
    img[(patch * 2) * per + pix] = (float)(s[2 * dof] * inv);
    img[(patch * 2 + 1) * per + pix] = (float)(s[2 * dof + 1] * inv);
}

// z += sigma * out, out on the coarse grid (f, nc; f = 1: the fine grid),
// spread piecewise constant
template <typename T>
__global__ void unpack_add_kernel(int64_t N, int n1, int f, int nc, const T* __restrict__ img,
                                  const double* __restrict__ ss, double* __restrict__ z) {
    int64_t dof = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (dof >= N) return;
    const int64_t per = (int64_t)n1 * n1, cper = (int64_t)nc * nc;
    const int64_t patch = dof / per, pix = dof % per;
    const int64_t cpix = (pix / n1 / f) * nc + (pix % n1) / f;
    const double sig = sqrt(ss[0] / (2.0 * N));
    z[2 * dof] += sig * (double)ld_act(img, (patch * 2) * cper + cpix);
    z[2 * dof + 1] += sig * (double)ld_act(img, (patch * 2 + 1) * cper + cpix);
}

__global__ void sumsq_kernel(int64_t n, const double* __restrict__ v, double* __restrict__ out) {
    __shared__ double red[1024];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += v[i] * v[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

namespace {

cudaError_t grow(void** p, size_t* have, size_t need_bytes) {
    if (need_bytes <= *have) return cudaSuccess;
    cudaFree(*p);
    *p = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc(p, need_bytes);
    if (!e) *have = need_bytes;
    return e;
}

cudaError_t ensure_buffers(ibem_cnn* c, int B, int H, int W) {
    int mc = 2;
    for (int l = 0; l < c->L; ++l) mc = std::max(mc, std::max(c->cin[l], c->cout[l]));
    const size_t slot = (size_t)B * mc * H * W;
    cudaError_t e;
    size_t ab = c->act_bytes;
    if ((e = grow(&c->d_act, &ab, slot * (c->L + 1) * sizeof(float)))) return e;
    c->act_bytes = ab;
    c->act_slot = slot;
    size_t gb = c->gbuf_floats * sizeof(float);
    if ((e = grow(reinterpret_cast<void**>(&c->d_gbuf), &gb, 2 * slot * sizeof(float)))) return e;
    c->gbuf_floats = gb / sizeof(float);
    return cudaSuccess;
}

template <typename TI, typename TO, typename TM>
void launch_conv(ibem_cnn* c, const TI* in, int B, int Cin, int H, int W, const float* w, const float* bias, int Cout,
                 int relu, int bf, const TM* mask, TO* out) {
    const int tiles = ((H + TS - 1) / TS) * ((W + TS - 1) / TS);
    if (Cout <= 4) {
        dim3 grid(tiles, 1, B);
        conv_tile_kernel<TI, TO, TM, 4><<<grid, 256, 0, c->stream>>>(in, Cin, H, W, w, bias, Cout, relu, bf, mask, out);
    } else {
        dim3 grid(tiles, (Cout + 15) / 16, B);
        conv_tile_kernel<TI, TO, TM, 16><<<grid, 256, 0, c->stream>>>(in, Cin, H, W, w, bias, Cout, relu, bf, mask, out);
    }
    ++c->launches;
}

// forward: slot 0 = input (converted), slot l + 1 = output of layer l
template <typename T>
cudaError_t forward(ibem_cnn* c, const float* in, int B, int H, int W, int bf) {
    cudaError_t e;
    if ((e = ensure_buffers(c, B, H, W))) return e;
    const size_t per = c->act_slot;
    T* act = reinterpret_cast<T*>(c->d_act);
    const int64_t n0 = (int64_t)B * 2 * H * W;
    f32_to_act_kernel<T><<<cblk(n0, 256), 256, 0, c->stream>>>(n0, in, act);
    ++c->launches;
    for (int l = 0; l < c->L; ++l)
        launch_conv<T, T, T>(c, act + l * per, B, c->cin[l], H, W, c->d_param + c->woff[l], c->d_param + c->boff[l],
                             c->cout[l], l + 1 < c->L ? 1 : 0, bf, nullptr, act + (l + 1) * per);
    return cudaGetLastError();
}

// Inference forward in BF16 on the tensor cores (C = 32 and a band that fits in
// shared memory; otherwise the FMA path).  Slots: 0 the input as BF16 pixel-major
// 8-channel pixels, 1..3 hidden outputs (pixel-major), 4 the output (planar), so
// the output sits where forward() leaves it.
template <int CGI, int NP, int NOUT, bool OUT_PLANAR>
cudaError_t launch_tc(ibem_cnn* c, const __nv_bfloat16* in, int B, int H, int W, const __nv_bfloat16* wt,
                      const float* bias, int relu, __nv_bfloat16* out, int* status, long long wait_limit) {
    constexpr int KG = CGI < 2 ? 2 : CGI;
    const int P = W + 2, nb = TC_M * TC_MB + 2 * P + 2, nbp = ((nb + 7) & ~7) + 2;
    const size_t sm = (size_t)9 * (NP / 8) * KG * 128 + (size_t)KG * nbp * 16 + 16;
    auto kern = conv_tc_kernel<CGI, NP, NOUT, OUT_PLANAR>;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern))) return e;
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev))) return e;
    // resident CTAs per SM from shared memory (1 KB reserved per CTA), registers
    // and TMEM (512 columns, 32 * TC_MB per CTA)
    int per_sm = (int)std::min<size_t>(512 / (32 * TC_MB), (size_t)233472 / (sm + 1024));
    per_sm = std::min(per_sm, 65536 / std::max(1, fa.numRegs * 128));
    per_sm = std::max(per_sm, 1);
    const int64_t ntiles = (int64_t)B * (((int64_t)H * P + TC_M * TC_MB - 1) / (TC_M * TC_MB));
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)per_sm * nsm));
    kern<<<grid, 128, sm, c->stream>>>(in, B, H, W, wt, bias, relu, nbp, out, wait_limit, status);
    ++c->launches;
    return cudaGetLastError();
}

bool tc_fits(int W) {
    const int P = W + 2, nb = TC_M * TC_MB + 2 * P + 2, nbp = ((nb + 7) & ~7) + 2;
    return (size_t)9 * 4 * 4 * 128 + (size_t)4 * nbp * 16 + 16 <= 227 * 1024;
}

cudaError_t forward_infer(ibem_cnn* c, const float* in, int B, int H, int W, int* status, long long wait_limit) {
    if (c->C != 32 || c->L != 4 || !tc_fits(W)) return forward<__nv_bfloat16>(c, in, B, H, W, 1);
    cudaError_t e;
    if ((e = ensure_buffers(c, B, H, W))) return e;
    // weight tiles: layer 0 [9][4][2], layers 1, 2 [9][4][4], layer 3 [9][2][4] cores of 64 elements
    const size_t w0 = 9 * 4 * 2 * 64, w1 = 9 * 4 * 4 * 64, w3 = 9 * 2 * 4 * 64;
    if ((e = grow(&c->d_wtc, &c->wtc_bytes, (w0 + 2 * w1 + w3) * sizeof(__nv_bfloat16)))) return e;
    __nv_bfloat16* wt = reinterpret_cast<__nv_bfloat16*>(c->d_wtc);
    __nv_bfloat16* wl[4] = {wt, wt + w0, wt + w0 + w1, wt + w0 + 2 * w1};
    const int np[4] = {32, 32, 32, 16}, kg[4] = {2, 4, 4, 4};
    for (int l = 0; l < 4; ++l) {
        const int n = np[l] * 8 * kg[l] * 9;
        tc_weights_kernel<<<cblk(n, 256), 256, 0, c->stream>>>(c->d_param + c->woff[l], c->cin[l], c->cout[l], np[l],
                                                              kg[l], wl[l]);
    }
    const size_t per = c->act_slot;
    __nv_bfloat16* act = reinterpret_cast<__nv_bfloat16*>(c->d_act);
    const int64_t npx = (int64_t)B * H * W;
    pack8_kernel<<<cblk(npx, 256), 256, 0, c->stream>>>(npx, (int64_t)H * W, in, act);
    c->launches += 5;
    if ((e = launch_tc<1, 32, 32, false>(c, act, B, H, W, wl[0], c->d_param + c->boff[0], 1, act + per, status,
                                         wait_limit)))
        return e;
    for (int l = 1; l <= 2; ++l)
        if ((e = launch_tc<4, 32, 32, false>(c, act + l * per, B, H, W, wl[l], c->d_param + c->boff[l], 1,
                                             act + (l + 1) * per, status, wait_limit)))
            return e;
    return launch_tc<4, 16, 2, true>(c, act + 3 * per, B, H, W, wl[3], c->d_param + c->boff[3], 0, act + 4 * per,
                                     status, wait_limit);
}

// backward from the loss against target (forward must have run on the same
// batch); gradients into d_grad, loss into d_red[0]
template <typename T>
cudaError_t backward(ibem_cnn* c, const float* target, int B, int H, int W, int bf, const float* gout = nullptr) {
    const size_t per = c->act_slot;
    T* act = reinterpret_cast<T*>(c->d_act);
    // g0 is only read below (the ReLU mask is fused into the next gradient)
    float* g0 = gout ? const_cast<float*>(gout) : c->d_gbuf;
    float* g1 = c->d_gbuf + per;
    float* g2 = c->d_gbuf;
    const int64_t HW = (int64_t)H * W;
    const int tiles = ((H + TS - 1) / TS) * ((W + TS - 1) / TS);
    const int64_t items = (int64_t)B * tiles;
    const int nx = (int)std::min<int64_t>(items, WG_ITEMS);
    const int ipc = (int)((items + nx - 1) / nx);
    cudaError_t e;
    size_t maxw = 0;
    for (int l = 0; l < c->L; ++l) maxw = std::max(maxw, (size_t)c->cout[l] * c->cin[l] * 9);
    size_t pb = c->part_floats * sizeof(float);
    if ((e = grow(reinterpret_cast<void**>(&c->d_part), &pb, (size_t)nx * maxw * sizeof(float)))) return e;
    c->part_floats = pb / sizeof(float);
    if (!gout) {
        loss_kernel<T><<<1, 1024, 0, c->stream>>>((int64_t)B * 2 * HW, B, act + c->L * per, target, g0, c->d_red);
        ++c->launches;
    }
    for (int l = c->L - 1; l >= 0; --l) {
        const int Cin = c->cin[l], Cout = c->cout[l];
        // g0 = dL / d(pre-activation of layer l)
        dim3 wg(nx, (Cin + CIB - 1) / CIB);
        conv_wgrad_kernel<T><<<wg, 256, 0, c->stream>>>(g0, act + l * per, B, Cin, H, W, Cout, ipc, c->d_part);
        const int nw = Cout * Cin * 9;
        sum_rows_kernel<<<cblk(nw, 256), 256, 0, c->stream>>>(c->d_part, nx, nw, c->d_grad + c->woff[l]);
        bias_grad_kernel<<<Cout, 256, 0, c->stream>>>(g0, B, Cout, HW, c->d_grad + c->boff[l]);
        c->launches += 3;
        if (l > 0) {
            flip_weights_kernel<<<cblk(nw, 256), 256, 0, c->stream>>>(c->d_param + c->woff[l], Cin, Cout, bf, c->d_wt);
            // dL/d(pre-activation of layer l-1): through the flipped convolution, masked by ReLU'
            launch_conv<float, float, T>(c, g0, B, Cout, H, W, c->d_wt, nullptr, Cin, 0, 0, act + l * per, g1);
            c->launches += 1;
            // next input gradient goes to the buffer that is not g1 (the caller's gout is never written)
            float* nxt = (g1 == c->d_gbuf + per) ? g2 : c->d_gbuf + per;
            g0 = g1;
            g1 = nxt;
        }
    }
    return cudaGetLastError();
}

void adam(ibem_cnn* c, float lr) {
    c->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - (float)std::pow(0.9, (double)c->step);
    const float c2 = 1.0f - (float)std::pow(0.999, (double)c->step);
    adam_kernel<<<cblk((int64_t)c->nparam, 256), 256, 0, c->stream>>>(c->nparam, c->d_param, c->d_grad, c->d_m, c->d_v,
                                                                       lr, b1, b2, c1, c2, 1e-8f);
    ++c->launches;
}

bool dims_ok(int B, int H, int W) {
    return B >= 1 && H >= 1 && W >= 1 && B <= 65535 && (int64_t)H * W <= (1ll << 24);
}

}  // namespace

// ---- residual-norm objective: L = 1/(2 nb) sum_j |A (s_j + sigma_j net(s_j / sigma_j)) - r_j|^2 ----

// dst[j] = e^{i theta_j} src[items[j].src] (complex vectors of N dofs)
__global__ void rot_gather_vec_kernel(int nb, int64_t N, const TrainItem* __restrict__ items,
                                      const double* __restrict__ src, double* __restrict__ dst) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nb * N) return;
    const int j = (int)(idx / N);
    const int64_t i = idx % N;
    const TrainItem it = items[j];
    const double re = src[((int64_t)it.src * N + i) * 2], im = src[((int64_t)it.src * N + i) * 2 + 1];
    dst[idx * 2] = (double)it.c * re - (double)it.s * im;
    dst[idx * 2 + 1] = (double)it.s * re + (double)it.c * im;
}

// out[j] = |v_j|^2, one CTA per vector of n doubles
__global__ void vec_sumsq_kernel(int64_t n, const double* __restrict__ v, double* __restrict__ out) {
    __shared__ double red[256];
    const double* vj = v + (int64_t)blockIdx.x * n;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += vj[i] * vj[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// y_j -= r_j in place and out[j] = |y_j|^2; one CTA per vector of n doubles
__global__ void residual_sumsq_kernel(int64_t n, const double* __restrict__ r, double* __restrict__ y,
                                      double* __restrict__ out) {
    __shared__ double red[256];
    const int64_t o = (int64_t)blockIdx.x * n;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double d = y[o + i] - r[o + i];
        y[o + i] = d;
        acc += d * d;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// red[0] = sum_j part[j] / (2 nb); red[2] += sum_j part[j] / 2
__global__ void op_loss_kernel(int nb, const double* __restrict__ part, double* __restrict__ red) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int j = 0; j < nb; ++j) s += part[j];
    red[0] = s / (2.0 * nb);
    red[2] += s / 2.0;
}

__global__ void conj_kernel(int64_t n_complex, double* __restrict__ v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_complex) v[2 * i + 1] = -v[2 * i + 1];
}

// img[(j npatch + patch) 2 + c][pix] = s_j / sigma_j, sigma_j^2 = ss[j] / (2N)
__global__ void batch_pack_kernel(int nb, int64_t N, int n1, const double* __restrict__ s,
                                  const double* __restrict__ ss, float* __restrict__ img) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nb * N) return;
    const int j = (int)(idx / N);
    const int64_t dof = idx % N, per = (int64_t)n1 * n1, npatch = N / per;
    const int64_t patch = dof / per, pix = dof % per;
    const double inv = ss[j] > 0.0 ? 1.0 / sqrt(ss[j] / (2.0 * N)) : 0.0;
    const int64_t o = ((int64_t)j * npatch + patch) * 2 * per + pix;
    img[o] = (float)(s[idx * 2] * inv);
    img[o + per] = (float)(s[idx * 2 + 1] * inv);
}

// z_j = s_j + sigma_j P out_j (out on the coarse grid f, nc; piecewise constant P)
template <typename T>
__global__ void batch_unpack_kernel(int nb, int64_t N, int n1, int f, int nc, const T* __restrict__ out,
                                    const double* __restrict__ ss, const double* __restrict__ s,
                                    double* __restrict__ z) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nb * N) return;
    const int j = (int)(idx / N);
    const int64_t dof = idx % N, per = (int64_t)n1 * n1, npatch = N / per, cper = (int64_t)nc * nc;
    const int64_t patch = dof / per, pix = dof % per;
    const int64_t cpix = (pix / n1 / f) * nc + (pix % n1) / f;
    const double sig = sqrt(ss[j] / (2.0 * N));
    const int64_t o = ((int64_t)j * npatch + patch) * 2 * cper + cpix;
    z[idx * 2] = s[idx * 2] + sig * (double)ld_act(out, o);
    z[idx * 2 + 1] = s[idx * 2 + 1] + sig * (double)ld_act(out, o + cper);
}

// gimg = (sigma_j / nb) (Re, Im) g_j
__global__ void batch_grad_images_kernel(int nb, int64_t N, int n1, const double* __restrict__ g,
                                         const double* __restrict__ ss, float* __restrict__ gimg) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nb * N) return;
    const int j = (int)(idx / N);
    const int64_t dof = idx % N, per = (int64_t)n1 * n1, npatch = N / per;
    const int64_t patch = dof / per, pix = dof % per;
    const double f = sqrt(ss[j] / (2.0 * N)) / nb;
    const int64_t o = ((int64_t)j * npatch + patch) * 2 * per + pix;
    gimg[o] = (float)(f * g[idx * 2]);
    gimg[o + per] = (float)(f * g[idx * 2 + 1]);
}

namespace {

// Scratch of the objective: vectors R, S, Z, Y, G ([nb][2N] each), ss and
// part ([nb] each), images and their gradient.
struct OpScratch {
    double *R, *S, *Z, *Y, *G, *ss, *part;
    float *img, *gimg;
    float *cimg, *cgimg;   // the same on the coarse grid (coarsening factor > 1)
};

cudaError_t op_scratch(ibem_cnn* c, int nb, int64_t N, int64_t img_per_vec, OpScratch* o) {
    const size_t vec = (size_t)2 * N;
    const size_t nd = 5 * (size_t)nb * vec + 2 * (size_t)nb;
    const size_t nf = 4 * (size_t)nb * img_per_vec;
    cudaError_t e;
    if ((e = grow(&c->d_opvec, &c->opvec_bytes, nd * sizeof(double)))) return e;
    if ((e = grow(&c->d_opimg, &c->opimg_bytes, nf * sizeof(float)))) return e;
    double* d = reinterpret_cast<double*>(c->d_opvec);
    o->R = d;
    o->S = d + (size_t)nb * vec;
    o->Z = d + 2 * (size_t)nb * vec;
    o->Y = d + 3 * (size_t)nb * vec;
    o->G = d + 4 * (size_t)nb * vec;
    o->ss = d + 5 * (size_t)nb * vec;
    o->part = o->ss + nb;
    o->img = reinterpret_cast<float*>(c->d_opimg);
    o->gimg = o->img + (size_t)nb * img_per_vec;
    o->cimg = o->gimg + (size_t)nb * img_per_vec;
    o->cgimg = o->cimg + (size_t)nb * img_per_vec;
    return cudaSuccess;
}

// One evaluation of the objective on the nb vectors in o.R (unit norm), and
// with grad its gradient into c->d_grad; loss into d_red[0].  Runs on c->stream,
// which must be the handle's stream.
template <typename T>
cudaError_t op_batch(ibem_handle* h, ibem_cnn* c, const OpScratch& o, int nb, int bf, int op_prec, bool grad) {
    Plan& P = h->P;
    const int64_t N = P.N, vec = 2 * N;
    const int n1 = P.n1, npatch = P.npatch;
    cudaStream_t st = c->stream;
    cudaError_t e;
    const int f = c->coarse, nc = (n1 + f - 1) / f;
    const int64_t nch = (int64_t)nb * npatch * 2;
    for (int j = 0; j < nb; ++j) apply_block_jacobi(h, o.R + (size_t)j * vec, o.S + (size_t)j * vec);
    vec_sumsq_kernel<<<nb, 256, 0, st>>>(vec, o.S, o.ss);
    batch_pack_kernel<<<cblk((int64_t)nb * N, 256), 256, 0, st>>>(nb, N, n1, o.S, o.ss, o.img);
    if (f > 1)
        restrict_images_kernel<<<cblk(nch * nc * nc, 256), 256, 0, st>>>(nch, n1, f, nc, o.img, o.cimg, 1);
    c->launches += nb + 2 + (f > 1 ? 1 : 0);
    if ((e = forward<T>(c, f > 1 ? o.cimg : o.img, nb * npatch, nc, nc, bf))) return e;
    batch_unpack_kernel<T><<<cblk((int64_t)nb * N, 256), 256, 0, st>>>(
        nb, N, n1, f, nc, reinterpret_cast<const T*>(c->d_act) + c->L * c->act_slot, o.ss, o.S, o.Z);
    if ((e = apply_operator(h, o.Z, o.Y, nb, op_prec))) return e;
    residual_sumsq_kernel<<<nb, 256, 0, st>>>(vec, o.R, o.Y, o.part);
    op_loss_kernel<<<1, 32, 0, st>>>(nb, o.part, c->d_red);
    c->launches += 3;
    if (!grad) return cudaGetLastError();
    // A^H y = conj(A conj(y)): the Galerkin matrix of the symmetric kernel is complex symmetric
    conj_kernel<<<cblk((int64_t)nb * N, 256), 256, 0, st>>>((int64_t)nb * N, o.Y);
    if ((e = apply_operator(h, o.Y, o.G, nb, op_prec))) return e;
    conj_kernel<<<cblk((int64_t)nb * N, 256), 256, 0, st>>>((int64_t)nb * N, o.G);
    batch_grad_images_kernel<<<cblk((int64_t)nb * N, 256), 256, 0, st>>>(nb, N, n1, o.G, o.ss, o.gimg);
    if (f > 1)   // gradient of the coarse output: P^T, the block sums
        restrict_images_kernel<<<cblk(nch * nc * nc, 256), 256, 0, st>>>(nch, n1, f, nc, o.gimg, o.cgimg, 0);
    c->launches += 3 + (f > 1 ? 1 : 0);
    if ((e = backward<T>(c, nullptr, nb * npatch, nc, nc, bf, f > 1 ? o.cgimg : o.gimg))) return e;
    return cudaGetLastError();
}

ibem_status op_checks(ibem_handle* h, ibem_cnn* c) {
    if (!h || !c) return IBEM_ERR_ARG;
    if (!h->assembled) return IBEM_ERR_STATE;
    if (!h->helm) return IBEM_ERR_ARG;
    return IBEM_OK;
}

}  // namespace

// Learned preconditioner application z = s + sigma * net(s / sigma), s = B^-1 v
// (complex v, z of length N).  Runs on the handle's stream; no host sync.
cudaError_t cnn_precondition(ibem_handle* h, ibem_cnn* c, const double* v, double* z) {
    Plan& P = h->P;
    cudaStream_t keep = c->stream;
    c->stream = h->stream;
    const int B = P.npatch, n1 = P.n1;
    cudaError_t e = cudaSuccess;
    size_t ib = c->img_floats * sizeof(float);
    if ((e = grow(reinterpret_cast<void**>(&c->d_img), &ib, (size_t)B * 2 * n1 * n1 * sizeof(float)))) {
        c->stream = keep;
        return e;
    }
    c->img_floats = ib / sizeof(float);
    const int f = c->coarse, nc = (n1 + f - 1) / f;
    if (f > 1) {
        size_t cb = c->cimg_floats * sizeof(float);
        if ((e = grow(reinterpret_cast<void**>(&c->d_cimg), &cb, (size_t)B * 2 * nc * nc * sizeof(float)))) {
            c->stream = keep;
            return e;
        }
        c->cimg_floats = cb / sizeof(float);
    }
    apply_block_jacobi(h, v, z);
    sumsq_kernel<<<1, 1024, 0, h->stream>>>(2 * P.N, z, c->d_red + 1);
    pack_images_kernel<<<cblk(P.N, 256), 256, 0, h->stream>>>(P.N, n1, z, c->d_red + 1, c->d_img);
    if (f > 1)
        restrict_images_kernel<<<cblk((int64_t)B * 2 * nc * nc, 256), 256, 0, h->stream>>>((int64_t)B * 2, n1, f, nc,
                                                                                           c->d_img, c->d_cimg, 1);
    e = forward_infer(c, f > 1 ? c->d_cimg : c->d_img, B, nc, nc, h->d_status, h->wait_limit);
    if (!e) {
        unpack_add_kernel<__nv_bfloat16><<<cblk(P.N, 256), 256, 0, h->stream>>>(
            P.N, n1, f, nc, reinterpret_cast<const __nv_bfloat16*>(c->d_act) + c->L * c->act_slot, c->d_red + 1, z);
        e = cudaGetLastError();
    }
    h->launches += 4 + 1 + c->L + (f > 1 ? 1 : 0);
    c->stream = keep;
    return e;
}

}  // namespace ibem

using namespace ibem;

extern "C" {

ibem_status ibem_cnn_create(int channels, unsigned long long seed, void* cuda_stream, ibem_cnn** out) {
    if (!out || channels < 1 || channels > 32) return IBEM_ERR_ARG;
    *out = nullptr;
    ibem_cnn* c = new ibem_cnn();
    c->C = channels;
    c->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&c->device);
    c->cin = {2, channels, channels, channels};
    c->cout = {channels, channels, channels, 2};
    size_t off = 0, maxw = 0;
    for (int l = 0; l < c->L; ++l) {
        c->woff.push_back(off);
        off += (size_t)c->cout[l] * c->cin[l] * 9;
        maxw = std::max(maxw, (size_t)c->cout[l] * c->cin[l] * 9);
        c->boff.push_back(off);
        off += c->cout[l];
    }
    c->nparam = off;
    // He initialisation N(0, 2 / (9 cin)), the last layer scaled by 1/4 so that
    // the untrained correction is small; zero biases
    std::vector<float> p(off, 0.0f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < c->L; ++l) {
        std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / (9.0 * c->cin[l])) * (l + 1 == c->L ? 0.25 : 1.0));
        for (size_t i = 0; i < (size_t)c->cout[l] * c->cin[l] * 9; ++i) p[c->woff[l] + i] = (float)nd(rng);
    }
    if (cudaMalloc(&c->d_param, off * sizeof(float)) || cudaMalloc(&c->d_grad, off * sizeof(float)) ||
        cudaMalloc(&c->d_m, off * sizeof(float)) || cudaMalloc(&c->d_v, off * sizeof(float)) ||
        cudaMalloc(&c->d_wt, maxw * sizeof(float)) || cudaMalloc(&c->d_red, 8 * sizeof(double)) ||
        cudaMalloc(&c->d_status, sizeof(int))) {
        ibem_cnn_destroy(c);
        return IBEM_ERR_OOM;
    }
    if (cudaMemcpyAsync(c->d_param, p.data(), off * sizeof(float), cudaMemcpyHostToDevice, c->stream) ||
        cudaMemsetAsync(c->d_grad, 0, off * sizeof(float), c->stream) ||
        cudaMemsetAsync(c->d_m, 0, off * sizeof(float), c->stream) ||
        cudaMemsetAsync(c->d_v, 0, off * sizeof(float), c->stream) ||
        cudaMemsetAsync(c->d_red, 0, 8 * sizeof(double), c->stream) ||
        cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream) || cudaStreamSynchronize(c->stream)) {
        ibem_cnn_destroy(c);
        return IBEM_ERR_CUDA;
    }
    *out = c;
    return IBEM_OK;
}

ibem_status ibem_cnn_set_coarsening(ibem_cnn* c, int factor) {
    if (!c || factor < 1 || factor > 64) return IBEM_ERR_ARG;
    c->coarse = factor;
    return IBEM_OK;
}

ibem_status ibem_cnn_destroy(ibem_cnn* c) {
    if (!c) return IBEM_OK;
    cudaStreamSynchronize(c->stream);
    cudaFree(c->d_param);
    cudaFree(c->d_grad);
    cudaFree(c->d_m);
    cudaFree(c->d_v);
    cudaFree(c->d_wt);
    cudaFree(c->d_act);
    cudaFree(c->d_gbuf);
    cudaFree(c->d_part);
    cudaFree(c->d_img);
    cudaFree(c->d_cimg);
    cudaFree(c->d_items);
    cudaFree(c->d_opvec);
    cudaFree(c->d_opimg);
    cudaFree(c->d_wtc);
    cudaFree(c->d_status);
    cudaFree(c->d_red);
    delete c;
    return IBEM_OK;
}

ibem_status ibem_cnn_params(ibem_cnn* c, float* get_host, const float* set_host, size_t* count) {
    if (!c) return IBEM_ERR_ARG;
    if (count) *count = c->nparam;
    cudaError_t e = cudaSuccess;
    if (set_host) {
        e = cudaMemcpyAsync(c->d_param, set_host, c->nparam * sizeof(float), cudaMemcpyHostToDevice, c->stream);
        // new parameters start a new optimisation
        if (!e) e = cudaMemsetAsync(c->d_m, 0, c->nparam * sizeof(float), c->stream);
        if (!e) e = cudaMemsetAsync(c->d_v, 0, c->nparam * sizeof(float), c->stream);
        c->step = 0;
    }
    if (!e && get_host)
        e = cudaMemcpyAsync(get_host, c->d_param, c->nparam * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    return e ? IBEM_ERR_CUDA : IBEM_OK;
}

ibem_status ibem_cnn_forward(ibem_cnn* c, const float* in_dev, int B, int H, int W, float* out_dev, int precision) {
    if (!c || !in_dev || !out_dev || !dims_ok(B, H, W)) return IBEM_ERR_ARG;
    if (precision != IBEM_FP32 && precision != IBEM_BF16) return IBEM_ERR_ARG;
    const int bf = precision == IBEM_BF16;
    cudaError_t e = bf ? forward_infer(c, in_dev, B, H, W, c->d_status, 1LL << 26) : forward<float>(c, in_dev, B, H, W, 0);
    if (e) return e == cudaErrorMemoryAllocation ? IBEM_ERR_OOM : IBEM_ERR_CUDA;
    const int64_t n = (int64_t)B * 2 * H * W;
    if (bf)
        act_to_f32_kernel<__nv_bfloat16><<<cblk(n, 256), 256, 0, c->stream>>>(
            n, reinterpret_cast<const __nv_bfloat16*>(c->d_act) + c->L * c->act_slot, out_dev);
    else
        act_to_f32_kernel<float><<<cblk(n, 256), 256, 0, c->stream>>>(
            n, reinterpret_cast<const float*>(c->d_act) + c->L * c->act_slot, out_dev);
    ++c->launches;
    return cudaGetLastError() ? IBEM_ERR_CUDA : IBEM_OK;
}

ibem_status ibem_cnn_gradients(ibem_cnn* c, const float* in_dev, const float* target_dev, int B, int H, int W,
                               int precision, float* grad_host, double* loss) {
    if (!c || !in_dev || !target_dev || !dims_ok(B, H, W)) return IBEM_ERR_ARG;
    if (precision != IBEM_FP32 && precision != IBEM_BF16) return IBEM_ERR_ARG;
    const int bf = precision == IBEM_BF16;
    cudaError_t e;
    if (bf) {
        e = forward<__nv_bfloat16>(c, in_dev, B, H, W, 1);
        if (!e) e = backward<__nv_bfloat16>(c, target_dev, B, H, W, 1);
    } else {
        e = forward<float>(c, in_dev, B, H, W, 0);
        if (!e) e = backward<float>(c, target_dev, B, H, W, 0);
    }
    if (!e && grad_host)
        e = cudaMemcpyAsync(grad_host, c->d_grad, c->nparam * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (!e && loss) e = cudaMemcpyAsync(loss, c->d_red, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return e == cudaErrorMemoryAllocation ? IBEM_ERR_OOM : IBEM_ERR_CUDA;
    return IBEM_OK;
}

ibem_status ibem_cnn_train_step(ibem_cnn* c, const float* in_dev, const float* target_dev, int B, int H, int W,
                                float lr, int precision, double* loss) {
    if (!c || !in_dev || !target_dev || !dims_ok(B, H, W) || !(lr > 0.0f)) return IBEM_ERR_ARG;
    if (precision != IBEM_FP32 && precision != IBEM_BF16) return IBEM_ERR_ARG;
    const int bf = precision == IBEM_BF16;
    cudaError_t e;
    if (bf) {
        e = forward<__nv_bfloat16>(c, in_dev, B, H, W, 1);
        if (!e) e = backward<__nv_bfloat16>(c, target_dev, B, H, W, 1);
    } else {
        e = forward<float>(c, in_dev, B, H, W, 0);
        if (!e) e = backward<float>(c, target_dev, B, H, W, 0);
    }
    if (e) return e == cudaErrorMemoryAllocation ? IBEM_ERR_OOM : IBEM_ERR_CUDA;
    adam(c, lr);
    if (loss) {
        if (cudaMemcpyAsync(loss, c->d_red, sizeof(double), cudaMemcpyDeviceToHost, c->stream) ||
            cudaStreamSynchronize(c->stream))
            return IBEM_ERR_CUDA;
    }
    return cudaGetLastError() ? IBEM_ERR_CUDA : IBEM_OK;
}

ibem_status ibem_cnn_train(ibem_cnn* c, const float* in_dev, const float* target_dev, int n_images, int H, int W,
                           int batch, int epochs, float lr, unsigned long long seed, int augment,
                           double* last_epoch_loss) {
    if (!c || !in_dev || !target_dev || n_images < 1 || batch < 1 || epochs < 1 || !(lr > 0.0f) ||
        !dims_ok(batch, H, W) || (augment & ~3))
        return IBEM_ERR_ARG;
    if ((augment & IBEM_AUGMENT_DIHEDRAL) && H != W) return IBEM_ERR_ARG;
    const int nb_max = std::min(batch, n_images);
    cudaError_t e;
    size_t ib = c->img_floats * sizeof(float);
    if ((e = grow(reinterpret_cast<void**>(&c->d_img), &ib, (size_t)2 * nb_max * 2 * H * W * sizeof(float))))
        return IBEM_ERR_OOM;
    c->img_floats = ib / sizeof(float);
    if ((e = grow(&c->d_items, &c->items_bytes, (size_t)n_images * sizeof(TrainItem)))) return IBEM_ERR_OOM;
    float* bin = c->d_img;
    float* btgt = c->d_img + (size_t)nb_max * 2 * H * W;
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> phase(0.0, 2.0 * M_PI);
    std::vector<TrainItem> items(n_images);
    std::vector<int> perm(n_images);
    TrainItem* d_items = reinterpret_cast<TrainItem*>(c->d_items);
    for (int ep = 0; ep < epochs; ++ep) {
        std::iota(perm.begin(), perm.end(), 0);
        std::shuffle(perm.begin(), perm.end(), rng);
        for (int i = 0; i < n_images; ++i) {
            const double th = (augment & IBEM_AUGMENT_PHASE) ? phase(rng) : 0.0;
            items[i].src = perm[i];
            items[i].dihedral = (augment & IBEM_AUGMENT_DIHEDRAL) ? (int)(rng() & 7) : 0;
            items[i].c = (float)std::cos(th);
            items[i].s = (float)std::sin(th);
        }
        // pageable copy: staged before return, ordered after the previous epoch
        if (cudaMemcpyAsync(d_items, items.data(), n_images * sizeof(TrainItem), cudaMemcpyHostToDevice, c->stream) ||
            cudaMemsetAsync(c->d_red + 2, 0, sizeof(double), c->stream))
            return IBEM_ERR_CUDA;
        for (int i0 = 0; i0 < n_images; i0 += nb_max) {
            const int nb = std::min(nb_max, n_images - i0);
            gather_kernel<<<cblk((int64_t)nb * H * W, 256), 256, 0, c->stream>>>(nb, H, W, d_items + i0, in_dev,
                                                                                 target_dev, bin, btgt);
            ++c->launches;
            e = forward<__nv_bfloat16>(c, bin, nb, H, W, 1);
            if (!e) e = backward<__nv_bfloat16>(c, btgt, nb, H, W, 1);
            if (e) return e == cudaErrorMemoryAllocation ? IBEM_ERR_OOM : IBEM_ERR_CUDA;
            adam(c, lr);
        }
    }
    double s = 0.0;
    if (cudaMemcpyAsync(&s, c->d_red + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream) ||
        cudaStreamSynchronize(c->stream))
        return IBEM_ERR_CUDA;
    // d_red[2] sums (1/2) |out - target|^2 over the images of the last epoch
    if (last_epoch_loss) *last_epoch_loss = s / n_images;
    return cudaGetLastError() ? IBEM_ERR_CUDA : IBEM_OK;
}

ibem_status ibem_cnn_operator_gradients(ibem_handle* h, ibem_cnn* c, const double* r_dev, int n, int precision,
                                        int op_precision, float* grad_host, double* loss) {
    ibem_status s = op_checks(h, c);
    if (s) return s;
    if (!r_dev || n < 1 || n > 256 || (precision != IBEM_FP32 && precision != IBEM_BF16) ||
        (op_precision != IBEM_FP64 && op_precision != IBEM_FP32))
        return IBEM_ERR_ARG;
    if (op_precision == IBEM_FP64 && h->P.prm.fp64_coupling == IBEM_COUPLING_FP32_ONLY) return IBEM_ERR_STATE;
    Plan& P = h->P;
    cudaStream_t keep = c->stream;
    c->stream = h->stream;
    OpScratch o;
    cudaError_t e = op_scratch(c, n, P.N, (int64_t)P.npatch * 2 * P.n1 * P.n1, &o);
    if (!e) e = cudaMemcpyAsync(o.R, r_dev, (size_t)n * 2 * P.N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    if (!e) {
        if (precision == IBEM_BF16) e = op_batch<__nv_bfloat16>(h, c, o, n, 1, op_precision, true);
        else e = op_batch<float>(h, c, o, n, 0, op_precision, true);
    }
    if (!e && grad_host)
        e = cudaMemcpyAsync(grad_host, c->d_grad, c->nparam * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (!e && loss) e = cudaMemcpyAsync(loss, c->d_red, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    c->stream = keep;
    if (e) return e == cudaErrorMemoryAllocation ? IBEM_ERR_OOM : IBEM_ERR_CUDA;
    return IBEM_OK;
}

ibem_status ibem_cnn_train_operator(ibem_handle* h, ibem_cnn* c, const double* r_dev, int n, int batch, int epochs,
                                    float lr, unsigned long long seed, int augment, int op_precision,
                                    double* last_epoch_loss) {
    ibem_status s = op_checks(h, c);
    if (s) return s;
    if (!r_dev || n < 1 || batch < 1 || batch > 256 || epochs < 1 || !(lr > 0.0f) ||
        (augment & ~IBEM_AUGMENT_PHASE) || (op_precision != IBEM_FP64 && op_precision != IBEM_FP32))
        return IBEM_ERR_ARG;
    if (op_precision == IBEM_FP64 && h->P.prm.fp64_coupling == IBEM_COUPLING_FP32_ONLY) return IBEM_ERR_STATE;
    Plan& P = h->P;
    const int nb_max = std::min(batch, n);
    cudaStream_t keep = c->stream;
    c->stream = h->stream;
    auto finish = [&](ibem_status r) {
        c->stream = keep;
        return r;
    };
    OpScratch o;
    cudaError_t e = op_scratch(c, nb_max, P.N, (int64_t)P.npatch * 2 * P.n1 * P.n1, &o);
    if (!e) e = grow(&c->d_items, &c->items_bytes, (size_t)n * sizeof(TrainItem));
    if (e) return finish(IBEM_ERR_OOM);
    TrainItem* d_items = reinterpret_cast<TrainItem*>(c->d_items);
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> phase(0.0, 2.0 * M_PI);
    std::vector<TrainItem> items(n);
    std::vector<int> perm(n);
    for (int ep = 0; ep < epochs; ++ep) {
        std::iota(perm.begin(), perm.end(), 0);
        std::shuffle(perm.begin(), perm.end(), rng);
        for (int i = 0; i < n; ++i) {
            const double th = (augment & IBEM_AUGMENT_PHASE) ? phase(rng) : 0.0;
            items[i] = TrainItem{perm[i], 0, (float)std::cos(th), (float)std::sin(th)};
        }
        if (cudaMemcpyAsync(d_items, items.data(), n * sizeof(TrainItem), cudaMemcpyHostToDevice, c->stream) ||
            cudaMemsetAsync(c->d_red + 2, 0, sizeof(double), c->stream))
            return finish(IBEM_ERR_CUDA);
        for (int i0 = 0; i0 < n; i0 += nb_max) {
            const int nb = std::min(nb_max, n - i0);
            rot_gather_vec_kernel<<<cblk((int64_t)nb * P.N, 256), 256, 0, c->stream>>>(nb, P.N, d_items + i0, r_dev,
                                                                                       o.R);
            ++c->launches;
            if ((e = op_batch<__nv_bfloat16>(h, c, o, nb, 1, op_precision, true)))
                return finish(e == cudaErrorMemoryAllocation ? IBEM_ERR_OOM : IBEM_ERR_CUDA);
            adam(c, lr);
        }
    }
    double sum = 0.0;
    if (cudaMemcpyAsync(&sum, c->d_red + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream) ||
        cudaStreamSynchronize(c->stream))
        return finish(IBEM_ERR_CUDA);
    if (last_epoch_loss) *last_epoch_loss = sum / n;
    return finish(cudaGetLastError() ? IBEM_ERR_CUDA : IBEM_OK);
}

ibem_status ibem_cnn_device_status(ibem_cnn* c, int* status) {
    if (!c || !status) return IBEM_ERR_ARG;
    if (cudaMemcpyAsync(status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream) ||
        cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream) || cudaStreamSynchronize(c->stream))
        return IBEM_ERR_CUDA;
    return IBEM_OK;
}

ibem_status ibem_cnn_launches(ibem_cnn* c, int64_t* launches) {
    if (!c || !launches) return IBEM_ERR_ARG;
    *launches = c->launches;
    c->launches = 0;
    return IBEM_OK;
}

}  // extern "C"
