// Block-Jacobi preconditioner of libibem (Sec. 4 item 3 uses Jacobi; the
// block variant groups the dofs whose anchor element - the element (ju, jv)
// clamped to the mesh, i.e. the last element of the B-spline's support - lies in
// one cluster of level max(0, m - 2)).  Each block of T A_near T^T is formed
// from the stored near-field blocks on the GPU, inverted on the host (LU with
// partial pivoting, FP64), and applied as a dense block-diagonal product.
#include <cmath>
#include <complex>

#include "ibem_internal.cuh"

namespace ibem {

// One CTA per block: entries (i, j) of T A_near T^T on the block's dofs.
// CW = 1 (real) or 2 (complex, blocks of double2).
template <int CW>
__global__ void bj_entries_kernel(const int64_t* __restrict__ bptr, const int32_t* __restrict__ bdofs,
                                  const int64_t* __restrict__ eoff, int p, int ne1, const int64_t* __restrict__ nptr,
                                  const int32_t* __restrict__ nsrc, const double* __restrict__ blocks,
                                  const double* __restrict__ ext, double* __restrict__ out) {
    const int64_t blk = blockIdx.x;
    const int64_t d0 = bptr[blk];
    const int bs = (int)(bptr[blk + 1] - d0);
    const int pp = p + 1, nb = pp * pp, n1 = ne1 + p;
    const int64_t per = (int64_t)ne1 * ne1;
    for (int ent = threadIdx.x; ent < bs * bs; ent += blockDim.x) {
        const int i = ent / bs, j = ent % bs;
        const int64_t di = bdofs[d0 + i], dj = bdofs[d0 + j];
        const int patch = (int)(di / ((int64_t)n1 * n1));
        const int ri = (int)(di % ((int64_t)n1 * n1)), rj = (int)(dj % ((int64_t)n1 * n1));
        const int jvi = ri / n1, jui = ri % n1, jvj = rj / n1, juj = rj % n1;
        double acc[2] = {0.0, 0.0};
        if ((int)(dj / ((int64_t)n1 * n1)) == patch) {
            for (int iy = jvi - p; iy <= jvi; ++iy)
                for (int ix = jui - p; ix <= jui; ++ix) {
                    if (ix < 0 || iy < 0 || ix >= ne1 || iy >= ne1) continue;
                    const int64_t e = patch * per + morton2(ix, iy);
                    const double* cu = ext + ((int64_t)ix * pp + (jui - ix)) * pp;
                    const double* cv = ext + ((int64_t)iy * pp + (jvi - iy)) * pp;
                    for (int iy2 = jvj - p; iy2 <= jvj; ++iy2)
                        for (int ix2 = juj - p; ix2 <= juj; ++ix2) {
                            if (ix2 < 0 || iy2 < 0 || ix2 >= ne1 || iy2 >= ne1) continue;
                            const int64_t e2 = patch * per + morton2(ix2, iy2);
                            int64_t lo = nptr[e], hi = nptr[e + 1];
                            while (lo < hi) {
                                int64_t mid = (lo + hi) >> 1;
                                if (nsrc[mid] < e2) lo = mid + 1; else hi = mid;
                            }
                            if (lo >= nptr[e + 1] || nsrc[lo] != e2) continue;
                            const double* B = blocks + lo * nb * nb * CW;
                            const double* du = ext + ((int64_t)ix2 * pp + (juj - ix2)) * pp;
                            const double* dv = ext + ((int64_t)iy2 * pp + (jvj - iy2)) * pp;
                            for (int a = 0; a < nb; ++a) {
                                double ta = cu[a % pp] * cv[a / pp];
                                double row[2] = {0.0, 0.0};
                                for (int b = 0; b < nb; ++b) {
                                    double tb = du[b % pp] * dv[b / pp];
                                    for (int c = 0; c < CW; ++c) row[c] += B[(a * nb + b) * CW + c] * tb;
                                }
                                for (int c = 0; c < CW; ++c) acc[c] += ta * row[c];
                            }
                        }
                }
        }
        for (int c = 0; c < CW; ++c) out[(eoff[blk] + ent) * CW + c] = acc[c];
    }
}

// z[dof_i] = sum_j Binv[i][j] r[dof_j]; one CTA per block.
template <int CW>
__global__ void bj_apply_kernel(const int64_t* __restrict__ bptr, const int32_t* __restrict__ bdofs,
                                const int64_t* __restrict__ eoff, const double* __restrict__ inv,
                                const double* __restrict__ r, double* __restrict__ z) {
    const int64_t blk = blockIdx.x;
    const int64_t d0 = bptr[blk];
    const int bs = (int)(bptr[blk + 1] - d0);
    const double* Bi = inv + eoff[blk] * CW;
    for (int i = threadIdx.x; i < bs; i += blockDim.x) {
        double ar = 0.0, ai = 0.0;
        for (int j = 0; j < bs; ++j) {
            int64_t dj = bdofs[d0 + j];
            if (CW == 1) {
                ar += Bi[i * bs + j] * r[dj];
            } else {
                double br = Bi[2 * (i * bs + j)], bi = Bi[2 * (i * bs + j) + 1];
                double xr = r[2 * dj], xi = r[2 * dj + 1];
                ar += br * xr - bi * xi;
                ai += br * xi + bi * xr;
            }
        }
        int64_t di = bdofs[d0 + i];
        if (CW == 1) {
            z[di] = ar;
        } else {
            z[2 * di] = ar;
            z[2 * di + 1] = ai;
        }
    }
}

namespace {

// In-place inverse of a dense n x n matrix (row-major) by Gauss-Jordan with
// partial pivoting; T = double or std::complex<double>.  Returns false if singular.
template <typename T>
bool invert(int n, T* A) {
    std::vector<T> I((size_t)n * n, T(0));
    for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = T(1);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::abs(A[(size_t)r * n + c]) > std::abs(A[(size_t)piv * n + c])) piv = r;
        if (std::abs(A[(size_t)piv * n + c]) == 0.0) return false;
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
                std::swap(I[(size_t)c * n + k], I[(size_t)piv * n + k]);
            }
        T d = A[(size_t)c * n + c];
        for (int k = 0; k < n; ++k) {
            A[(size_t)c * n + k] /= d;
            I[(size_t)c * n + k] /= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            T f = A[(size_t)r * n + c];
            if (f == T(0)) continue;
            for (int k = 0; k < n; ++k) {
                A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
                I[(size_t)r * n + k] -= f * I[(size_t)c * n + k];
            }
        }
    }
    std::copy(I.begin(), I.end(), A);
    return true;
}

}  // namespace

cudaError_t build_block_jacobi(ibem_handle* h, std::string* err) {
    Plan& P = h->P;
    const int lb = P.m >= 2 ? P.m - 2 : 0, shift = P.m - lb;
    const int64_t nper = (int64_t)1 << (2 * lb);
    const int64_t nblocks = P.npatch * nper;
    std::vector<std::vector<int32_t>> members(nblocks);
    for (int64_t dof = 0; dof < P.N; ++dof) {
        int patch = (int)(dof / ((int64_t)P.n1 * P.n1));
        int rem = (int)(dof % ((int64_t)P.n1 * P.n1));
        int jv = rem / P.n1, ju = rem % P.n1;
        int ax = ju < P.ne1 ? ju : P.ne1 - 1, ay = jv < P.ne1 ? jv : P.ne1 - 1;
        int64_t b = patch * nper + (int64_t)(ay >> shift) * ((int64_t)1 << lb) + (ax >> shift);
        members[b].push_back((int32_t)dof);
    }
    std::vector<int64_t> bptr(nblocks + 1, 0), eoff(nblocks + 1, 0);
    std::vector<int32_t> bdofs;
    for (int64_t b = 0; b < nblocks; ++b) {
        bptr[b + 1] = bptr[b] + (int64_t)members[b].size();
        eoff[b + 1] = eoff[b] + (int64_t)members[b].size() * (int64_t)members[b].size();
        bdofs.insert(bdofs.end(), members[b].begin(), members[b].end());
    }
    const int CW = h->helm ? 2 : 1;
    const int64_t nent = eoff[nblocks];
    cudaError_t e;
    cudaStream_t st = h->stream;
    if ((e = cudaMalloc(&h->d_bj_ptr, bptr.size() * sizeof(int64_t)))) return e;
    if ((e = cudaMalloc(&h->d_bj_off, eoff.size() * sizeof(int64_t)))) return e;
    if ((e = cudaMalloc(&h->d_bj_dofs, bdofs.size() * sizeof(int32_t)))) return e;
    if ((e = cudaMalloc(&h->d_bj_inv, (size_t)nent * CW * sizeof(double)))) return e;
    cudaMemcpyAsync(h->d_bj_ptr, bptr.data(), bptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->d_bj_off, eoff.data(), eoff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->d_bj_dofs, bdofs.data(), bdofs.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (CW == 1)
        bj_entries_kernel<1><<<(unsigned)nblocks, 128, 0, st>>>(h->d_bj_ptr, h->d_bj_dofs, h->d_bj_off, P.p, P.ne1,
                                                               h->d_near_ptr, h->d_near_src, h->d_near, h->d_ext,
                                                               h->d_bj_inv);
    else
        bj_entries_kernel<2><<<(unsigned)nblocks, 128, 0, st>>>(h->d_bj_ptr, h->d_bj_dofs, h->d_bj_off, P.p, P.ne1,
                                                               h->d_near_ptr, h->d_near_src, h->d_near, h->d_ext,
                                                               h->d_bj_inv);
    if ((e = cudaGetLastError())) return e;
    std::vector<double> ent((size_t)nent * CW);
    if ((e = cudaMemcpyAsync(ent.data(), h->d_bj_inv, ent.size() * sizeof(double), cudaMemcpyDeviceToHost, st)))
        return e;
    if ((e = cudaStreamSynchronize(st))) return e;
    for (int64_t b = 0; b < nblocks; ++b) {
        int n = (int)(bptr[b + 1] - bptr[b]);
        if (n == 0) continue;
        bool ok;
        if (CW == 1) ok = invert<double>(n, ent.data() + eoff[b]);
        else ok = invert<std::complex<double>>(n, reinterpret_cast<std::complex<double>*>(ent.data()) + eoff[b]);
        if (!ok) {
            *err = "block-Jacobi: singular diagonal block";
            return cudaErrorInvalidValue;
        }
    }
    if ((e = cudaMemcpyAsync(h->d_bj_inv, ent.data(), ent.size() * sizeof(double), cudaMemcpyHostToDevice, st)))
        return e;
    h->bj_blocks = nblocks;
    return cudaStreamSynchronize(st);
}

void apply_block_jacobi(ibem_handle* h, const double* r, double* z) {
    if (h->helm)
        bj_apply_kernel<2><<<(unsigned)h->bj_blocks, 64, 0, h->stream>>>(h->d_bj_ptr, h->d_bj_dofs, h->d_bj_off,
                                                                        h->d_bj_inv, r, z);
    else
        bj_apply_kernel<1><<<(unsigned)h->bj_blocks, 64, 0, h->stream>>>(h->d_bj_ptr, h->d_bj_dofs, h->d_bj_off,
                                                                        h->d_bj_inv, r, z);
}

}  // namespace ibem
