"""Right-hand side, solvers and potential evaluation (oracle; test only).

* Eq. varformdisc / Sec. 3.2: b_i = <g, b_i> = sum_e int k g(F) b_i (Gauss).
* Sec. 4 item 3: conjugate gradients for Laplace, GMRES for Helmholtz; here
  also a dense direct solve (numpy.linalg.solve) as the plain definition of the
  discrete solution.  Stopping rule (reading): true relative residual
  |b - A w| / |b| <= rtol.
* Eq. repform: u(x) = V~(w)(x) = int_Gamma u*(x, y) w(y) dy, evaluated with the
  same n x n Gauss rule per element as the right-hand side.

Pinned by: interior Laplace with a point source outside the sphere (u = g in
the ball) and exterior Helmholtz with a point source inside (u = g outside),
and CG / GMRES against the direct solve (tests/test_oracle_solve.py);
flexible GMRES by one step with the exact inverse, by equality with GMRES for a
fixed preconditioner and by convergence with a varying one
(tests/test_oracle_cnn.py).
"""
import numpy as np

from .galerkin import fundamental_solution


def dense_solve(A, b):
    return np.linalg.solve(A, b)


def cg(apply_A, b, rtol=1e-8, maxit=1000, diag=None):
    """Jacobi-preconditioned conjugate gradients for one right-hand side."""
    x = np.zeros_like(b)
    r = b.copy()
    z = r / diag if diag is not None else r.copy()
    p = z.copy()
    rz = np.vdot(r, z).real
    nb = np.linalg.norm(b)
    for it in range(1, maxit + 1):
        Ap = apply_A(p)
        alpha = rz / np.vdot(p, Ap).real
        x += alpha * p
        r -= alpha * Ap
        if np.linalg.norm(r) <= rtol * nb:
            return x, it
        z = r / diag if diag is not None else r.copy()
        rz_new = np.vdot(r, z).real
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit


def gmres(apply_A, b, rtol=1e-8, restart=100, maxit=1000, diag=None):
    """Right-preconditioned restarted GMRES (Jacobi), Arnoldi with two passes of
    classical Gram-Schmidt."""
    n = b.shape[0]
    dt = np.result_type(b, np.complex128)
    x = np.zeros(n, dtype=dt)
    nb = np.linalg.norm(b)
    Minv = (lambda v: v / diag) if diag is not None else (lambda v: v)
    total = 0
    while total < maxit:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        if beta <= rtol * nb:
            return x, total
        V = np.zeros((n, restart + 1), dtype=dt)
        H = np.zeros((restart + 1, restart), dtype=dt)
        V[:, 0] = r / beta
        k_done = 0
        for k in range(restart):
            w = apply_A(Minv(V[:, k]))
            for _ in range(2):
                h = V[:, :k + 1].conj().T @ w
                w = w - V[:, :k + 1] @ h
                H[:k + 1, k] += h
            H[k + 1, k] = np.linalg.norm(w)
            k_done = k + 1
            total += 1
            e1 = np.zeros(k + 2, dtype=dt)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:k + 2, :k + 1], e1, rcond=None)
            res = np.linalg.norm(H[:k + 2, :k + 1] @ y - e1)
            if H[k + 1, k].real == 0.0 or res <= rtol * nb or total >= maxit:
                break
            V[:, k + 1] = w / H[k + 1, k]
        x = x + Minv(V[:, :k_done] @ y)
    return x, total


def potential(disc, w, points):
    """u(x) = sum_e sum_qp (weight * k) u*(x, F_qp) w_h(qp) at points (P, 3)."""
    me = disc.mesh
    w2 = w.reshape(me.n_dofs, -1)
    dt = np.result_type(w2, np.complex128 if disc.kernel.is_complex else np.float64)
    u = np.zeros((len(points), w2.shape[1]), dtype=dt)
    for e in range(me.n_elements):
        _, F, k, wq, b, _ = disc._product_points(e, "regular")
        dens = b @ w2[me.local_dofs(e)]                                  # (nq, R)
        U = fundamental_solution(disc.kernel, points[:, None, :], F[None, :, :])
        u += U @ ((wq * k)[:, None] * dens)
    return u


def fgmres(apply_A, b, precond, rtol=1e-8, restart=100, maxit=1000, record=None):
    """Flexible GMRES (Saad, SIAM J. Sci. Comput. 14, 1993): right
    preconditioning where the preconditioner may change from step to step, so
    the preconditioned vectors z_k = precond(v_k) are kept and the iterate is
    x = x0 + Z y.  Arnoldi with two passes of classical Gram-Schmidt; the
    small least-squares problem is solved by numpy.linalg.lstsq.

    With ``record`` a list, the iterate x_k after every step of the first cycle
    is appended to it (used to form residual/error training pairs)."""
    n = b.shape[0]
    dt = np.result_type(b, np.complex128)
    x = np.zeros(n, dtype=dt)
    nb = np.linalg.norm(b)
    total = 0
    cycle = 0
    while total < maxit:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        if beta <= rtol * nb:
            return x, total
        V = np.zeros((n, restart + 1), dtype=dt)
        Z = np.zeros((n, restart), dtype=dt)
        H = np.zeros((restart + 1, restart), dtype=dt)
        V[:, 0] = r / beta
        k_done = 0
        for k in range(restart):
            Z[:, k] = precond(V[:, k])
            w = apply_A(Z[:, k])
            for _ in range(2):
                h = V[:, :k + 1].conj().T @ w
                w = w - V[:, :k + 1] @ h
                H[:k + 1, k] += h
            H[k + 1, k] = np.linalg.norm(w)
            k_done = k + 1
            total += 1
            e1 = np.zeros(k + 2, dtype=dt)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:k + 2, :k + 1], e1, rcond=None)
            if record is not None and cycle == 0:
                record.append(x + Z[:, :k + 1] @ y)
            res = np.linalg.norm(H[:k + 2, :k + 1] @ y - e1)
            if H[k + 1, k].real == 0.0 or res <= rtol * nb or total >= maxit:
                break
            V[:, k + 1] = w / H[k + 1, k]
        x = x + Z[:, :k_done] @ y
        cycle += 1
    return x, total
