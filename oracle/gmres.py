"""Right-preconditioned restarted GMRES (modified Gram-Schmidt, Givens rotations).

Oracle (test infrastructure only).

Paper: Sec. 6.1 -- the right-preconditioned system A B^{-1} u = b, x = B^{-1} u,
is solved by GMRES; stopping on a relative residual reduction; at most 200
iterations. Sec. 5.2 recalls GMRES as the minimal-residual Krylov method.

Readings:
  * initial guess x0 = 0 (the paper uses a random x0), so the relative residual
    is ||b - A x|| / ||b|| in the Euclidean norm (right preconditioning leaves the
    residual unpreconditioned);
  * restart length m (0 = unrestarted); at a restart x is formed and the true
    residual b - A x is recomputed;
  * Arnoldi by modified Gram-Schmidt; the small least-squares problem by complex
    Givens rotations (Saad, Iterative Methods, Alg. 6.9 and Prop. 6.9).
  * weighted GMRES (Sec. 5.2): with a Hermitian positive definite weight D, the Arnoldi
    process runs in <v, w>_D = w^* D v and the residual is minimised in ||.||_D; the
    stopping test is then on ||b - A x||_D / ||b||_D. The paper's weight is
    D_k = K + k^2 M, the matrix of the (.,.)_{curl,k} inner product (Eq. 2.3, Eq. 5.1).
  * flexible GMRES (Saad, SIAM J. Sci. Comput. 14 (1993), FGMRES): the preconditioned
    vectors z_j = B_j^{-1} v_j are kept and the iterate is x0 + Z_m y, which stays the
    minimal-residual solution over span(Z_m) when the preconditioner changes from one
    iteration to the next -- as it does when the coarse problem is solved only roughly by
    an inner iteration (Sec. 6.4). With a fixed preconditioner it equals GMRES.
"""
import numpy as np


def givens(a, b):
    """Complex rotation (c real, s complex) with [c s; -conj(s) c] [a; b] = [r; 0]."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, np.conj(b) / abs(b)
    t = np.hypot(abs(a), abs(b))
    c = abs(a) / t
    s = (a / abs(a)) * np.conj(b) / t
    return c, s


def gmres(matvec, precond, b, tol=1e-6, restart=0, max_it=200, x0=None, history=None, weight=None,
          flexible=False, arnoldi=None):
    """Solve A x = b with right preconditioner B^{-1}.

    matvec(v) = A v, precond(v) = B^{-1} v for 1-D complex vectors; weight(v) = D v for
    weighted GMRES (None: the Euclidean inner product); flexible: keep Z_m (FGMRES).
    arnoldi: a list that receives, per restart cycle, a dict of copies of the basis V_{k+1},
    the preconditioned vectors Z_k and the Hessenberg matrix before the rotations (H-bar_k),
    for checking the Arnoldi relation A Z_k = V_{k+1} H-bar_k.
    Returns (x, iterations, final relative true residual, converged)."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    D = weight if weight is not None else (lambda v: v)

    def dot(u, v):  # <v, u>_D = u^* D v (first argument conjugated, like np.vdot)
        return np.vdot(u, D(v))

    def norm(v):
        return float(np.sqrt(max(dot(v, v).real, 0.0)))

    bnorm = norm(b)
    if bnorm == 0.0:
        return np.zeros(n, dtype=np.complex128), 0, 0.0, True
    m = restart if restart > 0 else max_it
    its = 0
    r = b - matvec(x) if np.any(x) else b.copy()
    beta = norm(r)
    if beta / bnorm <= tol:
        return x, 0, beta / bnorm, True
    while True:
        V = np.zeros((m + 1, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        Z = np.zeros((m, n), dtype=np.complex128) if (flexible or arnoldi is not None) else None
        Hbar = np.zeros((m + 1, m), dtype=np.complex128) if arnoldi is not None else None
        j_done = 0
        converged = False
        for j in range(m):
            z = precond(V[j])
            if Z is not None:
                Z[j] = z
            w = matvec(z)
            for i in range(j + 1):  # modified Gram-Schmidt
                H[i, j] = dot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            if Hbar is not None:
                Hbar[:j + 2, j] = H[:j + 2, j]
            for i in range(j):  # previous rotations on the new column
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hi1
                H[i + 1, j] = -np.conj(sn[i]) * hi + cs[i] * hi1
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            if history is not None:
                history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or its >= max_it:
                converged = abs(g[j + 1]) / bnorm <= tol
                break
        k = j_done
        if arnoldi is not None:
            arnoldi.append({"V": V[:k + 1].copy(), "Z": Z[:k].copy(), "Hbar": Hbar[:k + 1, :k].copy()})
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])  # upper-triangular back substitution
        x = x + (Z[:k].T @ y if flexible else precond(V[:k].T @ y))
        r = b - matvec(x)
        beta = norm(r)
        rel = beta / bnorm
        if rel <= tol:
            return x, its, rel, True
        if its >= max_it:
            return x, its, rel, False
