"""Deflated preconditioned CG with a recycled Ritz space (oracle; test
infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this module).

Not in the paper, which solves its problem without a preconditioner; it
serves the Tikhonov CG solve E x = b of the reconstruction problem, E
Hermitian positive definite.  Published methods restated here:

  * Preconditioned CG (Hestenes-Stiefel with a Hermitian positive-definite
    preconditioner M, z = M r) and its Lanczos connection (Golub and Van Loan,
    "Matrix Computations", the CG-Lanczos relation; Saad, "Iterative Methods
    for Sparse Linear Systems", section 6.7.3): with alpha_j the step sizes,
    rho_j = <r_j, z_j> and beta_j = rho_{j+1} / rho_j, the vectors
    v_j = z_j / sqrt(rho_j) satisfy v_i^H M^-1 v_j = delta_ij and
        M E V_m = V_m T_m + (last column term),  T_m = V_m^H E V_m,
    T_m symmetric tridiagonal with
        T[j, j] = 1 / alpha_j + beta_{j-1} / alpha_{j-1}   (second term for j > 0)
        T[j, j+1] = T[j+1, j] = -sqrt(beta_j) / alpha_j
    (the off-diagonal sign belongs to these v_j; the Lanczos vectors of the
    usual statement are (-1)^j v_j, for which it is +: the same spectrum,
    eigenvectors that differ in the sign of every odd component).
    The eigenpairs (theta_i, s_i) of T_m give Ritz pairs (theta_i, V_m s_i) of
    M E; the smallest Ritz values approximate the smallest eigenvalues of M E.
  * Deflation (Tang, Nabben and Vuik, "Comparison of two-level preconditioners
    derived from deflation, domain decomposition and multigrid methods",
    J. Sci. Comput. 39 (2009), the A-DEF2 variant): with a basis W of k
    vectors, E_c = W^H E W, Q = W E_c^-1 W^H and P^T = I - Q E (E_c^-1 read as
    the Moore-Penrose inverse, so a nearly dependent W deflates its span),
        x_0 = Q b + P^T x_init,   r_0 = b - E x_0,   z_0 = M r_0,   p_0 = P^T z_0,
        alpha_j = <r_j, z_j> / <p_j, E p_j>,
        x_{j+1} = x_j + alpha_j p_j,   r_{j+1} = r_j - alpha_j E p_j,
        z_{j+1} = M r_{j+1},   beta_j = <r_{j+1}, z_{j+1}> / <r_j, z_j>,
        p_{j+1} = P^T z_{j+1} + beta_j p_j.
    Every residual satisfies W^H r_j = 0 and every direction W^H E p_j = 0,
    so the iteration runs on the spectrum of M E with W's part removed.

Inner products of the complex system are taken as real parts where the
equivalent real symmetric system needs them (alpha, beta, rho), complex
where a projection coefficient is formed (W^H v).
"""

from __future__ import annotations

import numpy as np


def _dot_re(a, b):
    return float(np.vdot(a, b).real)


def pcg_record(apply_E, apply_M, b, tol: float = 1e-4, maxit: int = 100, record: int = 0):
    """Preconditioned CG from x = 0 on E x = b with z = M r.  Returns (x,
    iterations, relative residual history, alphas, rhos, Z) where rhos[j] =
    <r_j, z_j> and Z holds z_j / sqrt(rho_j) for the first `record` steps
    (the Lanczos vectors of M E)."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    r = b.copy()
    z = apply_M(r)
    p = z.copy()
    rho = _dot_re(r, z)
    bnorm = np.sqrt(_dot_re(b, b))
    hist = [np.sqrt(_dot_re(r, r)) / bnorm if bnorm > 0 else 0.0]
    alphas, rhos, Z = [], [rho], []
    it = 0
    while it < maxit and hist[-1] > tol:
        if len(Z) < record:
            Z.append(z / np.sqrt(rho))
        Ep = apply_E(p)
        alpha = rho / _dot_re(p, Ep)
        x = x + alpha * p
        r = r - alpha * Ep
        z = apply_M(r)
        rho_new = _dot_re(r, z)
        p = z + (rho_new / rho) * p
        rho = rho_new
        alphas.append(alpha)
        rhos.append(rho)
        it += 1
        hist.append(np.sqrt(_dot_re(r, r)) / bnorm)
    return x, it, np.asarray(hist), np.asarray(alphas), np.asarray(rhos), Z


def lanczos_tridiagonal(alphas, rhos, m: int):
    """T_m = V_m^H E V_m of the CG-Lanczos relation (v_j = z_j / sqrt(rho_j))
    from the first m step sizes and the rho values (rhos[j] = <r_j, z_j>, at
    least m + 1 of them)."""
    a = np.asarray(alphas, dtype=np.float64)[:m]
    rho = np.asarray(rhos, dtype=np.float64)
    beta = rho[1:m + 1] / rho[:m]
    T = np.zeros((m, m))
    for j in range(m):
        T[j, j] = 1.0 / a[j] + (beta[j - 1] / a[j - 1] if j > 0 else 0.0)
        if j + 1 < m:
            T[j, j + 1] = T[j + 1, j] = -np.sqrt(beta[j]) / a[j]
    return T


def ritz_space(T, Z, k: int, largest: bool = False):
    """The k smallest (largest=True: largest, in descending order) Ritz values
    of T and their Ritz vectors sum_j s_i[j] Z[j]."""
    theta, S = np.linalg.eigh(T)
    m = T.shape[0]
    idx = list(range(m - 1, m - 1 - k, -1)) if largest else list(range(k))
    W = [sum(S[j, i] * Z[j] for j in range(m)) for i in idx]
    return theta[idx], W


def deflated_pcg(apply_E, apply_M, b, W, tol: float = 1e-4, maxit: int = 100, x_init=None):
    """A-DEF2 deflated preconditioned CG on E x = b with the basis W (a list
    of k vectors).  Returns (x, iterations, relative residual history,
    max_j |W^H r_j| / |b|)."""
    b = np.asarray(b, dtype=np.complex128)
    Wm = np.stack([np.asarray(w, dtype=np.complex128).reshape(-1) for w in W], 1)
    shape = b.shape
    EW = np.stack([apply_E(w.reshape(shape)).reshape(-1) for w in Wm.T], 1)
    Ec = Wm.conj().T @ EW
    # Moore-Penrose inverse (eigenvalues below 1e-10 of the largest dropped):
    # the deflation of span(W) when W is (nearly) rank-deficient, the inverse
    # otherwise
    Eci = np.linalg.pinv(Ec, rcond=1e-10, hermitian=True)

    def Q(v):
        return (Wm @ (Eci @ (Wm.conj().T @ v.reshape(-1)))).reshape(shape)

    def PT(v):  # v - W Ec^-1 (E W)^H v  (E Hermitian: W^H E v = (E W)^H v)
        return v - (Wm @ (Eci @ (EW.conj().T @ v.reshape(-1)))).reshape(shape)

    x = Q(b) if x_init is None else Q(b) + PT(np.asarray(x_init, dtype=np.complex128))
    r = b - apply_E(x)
    z = apply_M(r)
    p = PT(z)
    rho = _dot_re(r, z)
    bnorm = np.sqrt(_dot_re(b, b))
    hist = [np.sqrt(_dot_re(r, r)) / bnorm if bnorm > 0 else 0.0]
    wr = [np.linalg.norm(Wm.conj().T @ r.reshape(-1)) / bnorm]
    it = 0
    while it < maxit and hist[-1] > tol:
        Ep = apply_E(p)
        alpha = rho / _dot_re(p, Ep)
        x = x + alpha * p
        r = r - alpha * Ep
        z = apply_M(r)
        rho_new = _dot_re(r, z)
        p = PT(z) + (rho_new / rho) * p
        rho = rho_new
        it += 1
        hist.append(np.sqrt(_dot_re(r, r)) / bnorm)
        wr.append(np.linalg.norm(Wm.conj().T @ r.reshape(-1)) / bnorm)
    return x, it, np.asarray(hist), float(max(wr))
