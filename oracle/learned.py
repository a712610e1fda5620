"""Block-Jacobi and the learned right preconditioner built around it (oracle;
test infrastructure only).

Block-Jacobi (Sec. 4 item 3 names Jacobi; the block variant is a reading): the
dofs are grouped by the cluster of level max(0, m - 2) that holds their anchor
element, the element (min(ju, 2^m - 1), min(jv, 2^m - 1)) of the patch; each
diagonal block of the near-field matrix (the non-admissible element pairs of
the block cluster tree, Sec. 4.1) is inverted exactly.

Learned preconditioner (no counterpart in the paper): with s = B^-1 v the
block-Jacobi vector and sigma = |s| / sqrt(2 N) (the root mean square of its
real components), the network of ``oracle.cnn`` maps the patch images of
s / sigma to a correction, and
    z = s + sigma * net(s / sigma).
A training pair is built from a residual r and the error e with A e = r:
input s / sigma, target (e - s) / sigma, with s = B^-1 r.  The network thus
learns what block-Jacobi misses, in units that do not depend on the level, the
wavenumber or the size of r.

Operator-aware objective: the error of the preconditioned pair measured in the
residual norm, |A (z - e)| = |A z - r| with z = M(r), so that
    L = 1 / (2 nb) * sum_j |A M(r_j) - r_j|^2
over nb residuals of unit norm (e is not needed).  With z_j = s_j + sigma_j
net(x_j) and the complex linear A, dL / d(real, imag of z_j) is
A^H (A z_j - r_j) / nb, and dL / d(net output of x_j) is sigma_j times that,
in the real / imaginary channels.

Coarse-grid variant (coarsening factor f >= 1; f = 1 is the above): the
network sees each patch image averaged over blocks of f x f pixels (ragged
blocks at the far edge average the pixels they hold), R, and its output is
spread back over the blocks, P (piecewise constant):
    z = s + sigma * P net(R(s / sigma)).
The receptive field of the four 3 x 3 layers then spans 9 f pixels, so the
network can act on the smooth, patch-wide part of the error that block-Jacobi
leaves; with f = 2^(m - l) it always sees the level-l grid.  The gradient with
respect to the network output is P^T of the fine one (block sums).

Pinned by: the block groups cover every dof once and follow the anchor
elements, a network whose last layer is zero gives block-Jacobi exactly, z is
homogeneous of degree one in v, a training pair rebuilds e from its input and
target, and the gradient of the residual-norm objective against central
differences, with f = 1 and f = 2 on ragged images; R P is the identity and P
is the adjoint of the block sum (tests/test_oracle_cnn.py).
"""
import numpy as np

from . import cnn


def near_matrix(fmm):
    """Dense near-field matrix sum over near element pairs of their blocks."""
    me = fmm.mesh
    dt = np.complex128 if fmm.disc.kernel.is_complex else np.float64
    A = np.zeros((me.n_dofs, me.n_dofs), dtype=dt)
    for eA, eB in fmm.near_elements:
        dA, dB = me.local_dofs(eA), me.local_dofs(eB)
        A[np.ix_(dA, dB)] += fmm.near_block(eA, eB)
    return A


def block_jacobi_groups(mesh):
    """Dof index arrays of the blocks, in cluster order (patch, cy, cx)."""
    lb = max(0, mesh.m - 2)
    sh = mesh.m - lb
    n1, ne1 = mesh.n1, mesh.ne1
    groups = {}
    for dof in range(mesh.n_dofs):
        patch, rem = divmod(dof, n1 * n1)
        jv, ju = divmod(rem, n1)
        ax, ay = min(ju, ne1 - 1), min(jv, ne1 - 1)
        key = (patch, ay >> sh, ax >> sh)
        groups.setdefault(key, []).append(dof)
    return [np.array(groups[k]) for k in sorted(groups)]


class BlockJacobi:
    def __init__(self, Anear, groups):
        self.groups = groups
        self.inv = [np.linalg.inv(Anear[np.ix_(g, g)]) for g in groups]

    def __call__(self, v):
        z = np.zeros_like(v, dtype=np.result_type(v, self.inv[0]))
        for g, Bi in zip(self.groups, self.inv):
            z[g] = Bi @ v[g]
        return z


def rms(s):
    return np.linalg.norm(s) / np.sqrt(2.0 * s.shape[0])


def coarse_size(n1, f):
    return -(-n1 // f)


def restrict(img, f):
    """Mean over f x f pixel blocks: [B, c, n1, n1] -> [B, c, nc, nc]."""
    if f == 1:
        return img
    B, c, n1, _ = img.shape
    nc = coarse_size(n1, f)
    out = np.zeros((B, c, nc, nc))
    for Y in range(nc):
        for X in range(nc):
            blk = img[:, :, Y * f:(Y + 1) * f, X * f:(X + 1) * f]
            out[:, :, Y, X] = blk.mean(axis=(2, 3))
    return out


def prolong(img, f, n1):
    """Piecewise constant: fine pixel (y, x) takes coarse pixel (y // f, x // f)."""
    if f == 1:
        return img
    idx = np.arange(n1) // f
    return img[:, :, idx][:, :, :, idx]


def prolong_adjoint(img, f, nc):
    """P^T: sums over the f x f blocks."""
    if f == 1:
        return img
    B, c, n1, _ = img.shape
    out = np.zeros((B, c, nc, nc))
    for Y in range(nc):
        for X in range(nc):
            out[:, :, Y, X] = img[:, :, Y * f:(Y + 1) * f, X * f:(X + 1) * f].sum(axis=(2, 3))
    return out


def learned_apply(v, bj, params, C, n1, f=1):
    s = bj(v)
    sigma = rms(s)
    if sigma == 0.0:
        return s
    out = cnn.forward(params, restrict(cnn.vector_to_images(s / sigma, n1), f), C)
    return s + sigma * cnn.images_to_vector(prolong(out, f, n1))


def training_pair(r, e, bj, n1):
    """(input images, target images) of one residual/error pair."""
    s = bj(r)
    sigma = rms(s)
    return cnn.vector_to_images(s / sigma, n1), cnn.vector_to_images((e - s) / sigma, n1)


def operator_loss_and_grad(params, rs, apply_A, apply_AH, bj, C, n1, f=1):
    """L = 1/(2 nb) sum_j |A (s_j + sigma_j P net(R(s_j / sigma_j))) - r_j|^2 and
    dL/dparams for residuals rs [nb, N] (complex)."""
    nb = rs.shape[0]
    ss = [bj(r) for r in rs]
    sig = [rms(s) for s in ss]
    X = np.concatenate([restrict(cnn.vector_to_images(s / g, n1), f) for s, g in zip(ss, sig)])
    out, acts, pres = cnn.forward(params, X, C, keep=True)
    npatch = X.shape[0] // nb
    nc = coarse_size(n1, f)
    loss = 0.0
    gout = np.zeros_like(out)
    for j in range(nb):
        sl = slice(j * npatch, (j + 1) * npatch)
        z = ss[j] + sig[j] * cnn.images_to_vector(prolong(out[sl], f, n1))
        res = apply_A(z) - rs[j]
        loss += 0.5 * np.vdot(res, res).real / nb
        gout[sl] = sig[j] * prolong_adjoint(cnn.vector_to_images(apply_AH(res) / nb, n1), f, nc)
    return loss, cnn.backward(params, acts, pres, gout, C)
