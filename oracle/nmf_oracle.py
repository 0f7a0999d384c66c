"""Plain FP64 CPU oracle for beta-divergence NMF: joint MM (JMM) and block MM (BMM).

TEST INFRASTRUCTURE ONLY. This module exists to check the CUDA library against
the paper (Marmin, Goulart, Fevotte, "Joint Majorization-Minimization for
Nonnegative Matrix Factorization with the beta-divergence", arXiv 2106.15214).
Only the test suite, the smoke check and the CPU-baseline leg of the benchmark
may import it. The product path never calls it and shares no code with it.

Everything is numpy float64, written as whole-matrix expressions in the order
and notation of the paper. Matrix products use numpy's matmul (a library
primitive); there is no blocking, fusion or reassociation beyond what an
equation states.

Shapes: V is F x N, W is F x K, H is K x N (Sec. 2.1, eq. nmf).

Readings of points the paper leaves open:
  * 0 log 0 = 0 in the KL divergence (beta = 1), so d_1(0 | y) = y.
  * kappa (Sec. 4.1.3 "Handling zero values") is added to V and to every
    product WH that enters an update or the objective; default 0.
  * Normalisation (Sec. 4.1.2) divides each column of W by its l2 norm and
    multiplies the matching row of H by it; a zero column is left unchanged.
  * The mirrored update order ("H first") is the paper's remark that the order
    of the two updates in eq. jnt_update may be inverted (Sec. 4.1.1).
  * The gradient used by the KKT residuals (Sec. 4.1.5) is the gradient of
    D_beta(V + kappa | WH + kappa).
  * eps (the positivity constraint W, H >= eps under which eqs. Wll, Hll pose
    the block updates, Sec. 3.3.4): every update is clamped to eps, which is
    the constrained argmin of the per-entry convex auxiliary function; eps = 0
    (the default) is the unconstrained method.

Parity status of each function is stated in its docstring; every function here
is pinned by tests/test_oracle_pins.py (the gamma = 1 heuristic and BMM with
L_W, L_H > 1 by tests/test_oracle_variants.py) unless it says "parity
unpinned".
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gamma", "beta_divergence", "D_beta", "divergence_parts", "divergence_parts_dy",
    "chi1", "chi2", "auxiliary_G", "jmm_iteration", "bmm_iteration", "normalize",
    "run", "gradients", "kkt_residuals", "sparse_kl_jmm_iteration",
    "sparse_kl_bmm_iteration", "sparse_kl_objective", "sparse_kl_gradients",
    "batched_run",
]


# ---------------------------------------------------------------------------
# Scalars and the objective
# ---------------------------------------------------------------------------

def gamma(beta: float) -> float:
    """MM exponent gamma(beta), eq. def_gamma (Sec. 2.2)."""
    if beta < 1:
        return 1.0 / (2.0 - beta)
    if beta <= 2:
        return 1.0
    return 1.0 / (beta - 1.0)


def beta_divergence(x, y, beta: float):
    """Elementwise d_beta(x | y), eq. beta-div (Sec. 2.1).

    beta = 1: x log(x/y) - x + y (with 0 log 0 = 0); beta = 0: x/y - log(x/y) - 1;
    otherwise x^b / (b(b-1)) + y^b / b - x y^(b-1) / (b-1).
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if beta == 1:
        with np.errstate(divide="ignore", invalid="ignore"):
            xlog = np.where(x > 0, x * np.log(np.where(x > 0, x, 1.0) / y), 0.0)
        return xlog - x + y
    if beta == 0:
        r = x / y
        return r - np.log(r) - 1.0
    return (x ** beta / (beta * (beta - 1.0)) + y ** beta / beta
            - x * y ** (beta - 1.0) / (beta - 1.0))


def D_beta(V, WH, beta: float) -> float:
    """Objective D_beta(V | WH) = sum_fn d_beta(v_fn | [WH]_fn), eq. obj_fct.

    numpy's sum is pairwise, so the FP64 rounding error stays small.
    """
    return float(np.sum(beta_divergence(V, WH, beta)))


# ---------------------------------------------------------------------------
# Table 1: convex / concave / constant decomposition of d_beta in its 2nd arg
# ---------------------------------------------------------------------------

def divergence_parts(v, y, beta: float):
    """(convex, concave, constant) parts of d_beta(v | y) in y, Table 1."""
    v = np.asarray(v, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    zero = np.zeros(np.broadcast(v, y).shape)
    if beta < 1 and beta != 0:
        return (-v / (beta - 1.0) * y ** (beta - 1.0),
                y ** beta / beta + zero,
                v ** beta / (beta * (beta - 1.0)) + zero)
    if beta == 0:
        return v / y, np.log(y) + zero, -(np.log(v) + 1.0) + zero
    if beta <= 2:
        return beta_divergence(v, y, beta) + zero, zero, zero
    return (y ** beta / beta + zero,
            -v / (beta - 1.0) * y ** (beta - 1.0),
            v ** beta / (beta * (beta - 1.0)) + zero)


def divergence_parts_dy(v, y, beta: float):
    """Derivative in y of the concave part of Table 1 (used by the tangent bound)."""
    v = np.asarray(v, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if beta < 1 and beta != 0:
        return y ** (beta - 1.0) + 0.0 * v
    if beta == 0:
        return 1.0 / y + 0.0 * v
    if beta <= 2:
        return np.zeros(np.broadcast(v, y).shape)
    return -v * y ** (beta - 2.0)


# ---------------------------------------------------------------------------
# Joint auxiliary function G (Sec. 3.1)
# ---------------------------------------------------------------------------

def auxiliary_G(V, W, H, Wt, Ht, beta: float) -> float:
    """Joint majoriser G(W, H | Wt, Ht), eq. jointG.

    Convex part: Jensen with weights lambda_fnk = wt_fk ht_kn / vt_fn, eq. simplif.
    Concave part: tangent at vt_fn. Constant part: Table 1.
    """
    V = np.asarray(V, dtype=np.float64)
    Vt = Wt @ Ht
    lam = Wt[:, None, :] * Ht.T[None, :, :] / Vt[:, :, None]           # F x N x K
    arg = W[:, None, :] * H.T[None, :, :] / lam                          # w_fk h_kn / lam
    conv, _, _ = divergence_parts(V[:, :, None], arg, beta)
    G_conv = np.sum(lam * conv, axis=2)
    _, conc_t, const = divergence_parts(V, Vt, beta)
    G_conc = conc_t + divergence_parts_dy(V, Vt, beta) * (W @ H - Vt)
    return float(np.sum(G_conv + G_conc + const))


# ---------------------------------------------------------------------------
# JMM (Sec. 3.2, eq. jnt_update, Algorithm 2)
# ---------------------------------------------------------------------------

def chi1(X, Xt, beta: float):
    """chi_{1,beta}(X, Xt): Xt^(2-b) / X^(1-b) if b <= 2, else X (Sec. 3.2)."""
    if beta <= 2:
        return Xt ** (2.0 - beta) / X ** (1.0 - beta)
    return X.copy()


def chi2(X, Xt, beta: float):
    """chi_{2,beta}(X, Xt): X if b < 1, else X^b / Xt^(b-1) (Sec. 3.2)."""
    if beta < 1:
        return X.copy()
    return X ** beta / Xt ** (beta - 1.0)


def _floor(X, eps: float):
    """Entrywise max(X, eps): over x >= eps the minimiser of a convex function
    of one variable is its unconstrained minimiser clamped to eps, so this is
    the argmin of the auxiliary function under the constraint X >= eps
    (eqs. Wll, Hll). eps = 0 returns X unchanged."""
    return np.maximum(X, eps) if eps > 0 else X


def jmm_iteration(V, Wt, Ht, beta: float, L: int = 1, order: str = "W",
                  kappa: float = 0.0, gamma_one: bool = False, eps: float = 0.0):
    """One outer iteration of Algorithm 2 (JMM) from the iterate (Wt, Ht).

    Vt = Wt Ht is formed once (step "Vt <- Wt Ht"); then L inner passes each
    update W from chi(H_l, Ht) and H from chi(W_{l+1}, Wt), always rescaling
    Wt and Ht, eq. jnt_update. order="H" applies the two updates in the
    inverted order (Sec. 4.1.1 remark). kappa as in Sec. 4.1.3. gamma_one=True
    is the heuristic of Sec. 3.3.3 (gamma set to 1; oracle-only variant).
    eps > 0 clamps each update to eps (see _floor).
    Returns (W, H) before any normalisation.
    """
    g = 1.0 if gamma_one else gamma(beta)
    Vk = V + kappa
    Vt = Wt @ Ht + kappa
    A = Vk / Vt ** (2.0 - beta)          # V / Vt^(2-b)
    B = Vt ** (beta - 1.0)               # Vt^(b-1)
    W, H = Wt.copy(), Ht.copy()
    for _ in range(L):
        if order == "W":
            W = _floor(Wt * ((A @ chi1(H, Ht, beta).T) / (B @ chi2(H, Ht, beta).T)) ** g, eps)
            H = _floor(Ht * ((chi1(W, Wt, beta).T @ A) / (chi2(W, Wt, beta).T @ B)) ** g, eps)
        elif order == "H":
            H = _floor(Ht * ((chi1(W, Wt, beta).T @ A) / (chi2(W, Wt, beta).T @ B)) ** g, eps)
            W = _floor(Wt * ((A @ chi1(H, Ht, beta).T) / (B @ chi2(H, Ht, beta).T)) ** g, eps)
        else:
            raise ValueError(order)
    return W, H


# ---------------------------------------------------------------------------
# BMM (Sec. 2.2, eq. alt_update, Algorithm 1)
# ---------------------------------------------------------------------------

def _bmm_w_update(V, W, H, beta, g, kappa):
    WH = W @ H + kappa
    return W * ((((WH ** (beta - 2.0)) * (V + kappa)) @ H.T)
                / ((WH ** (beta - 1.0)) @ H.T)) ** g


def _bmm_h_update(V, W, H, beta, g, kappa):
    WH = W @ H + kappa
    return H * ((W.T @ ((WH ** (beta - 2.0)) * (V + kappa)))
                / (W.T @ (WH ** (beta - 1.0)))) ** g


def bmm_iteration(V, W, H, beta: float, LW: int = 1, LH: int = 1, order: str = "W",
                  kappa: float = 0.0, gamma_one: bool = False, eps: float = 0.0):
    """One outer iteration of Algorithm 1 (BMM): L_W updates of W with H fixed,
    then L_H updates of H with the new W fixed (eq. alt_update); the product
    WH is recomputed before every update. order="H" swaps the two blocks;
    eps > 0 clamps each update to eps (see _floor)."""
    g = 1.0 if gamma_one else gamma(beta)
    W, H = W.copy(), H.copy()
    if order == "W":
        for _ in range(LW):
            W = _floor(_bmm_w_update(V, W, H, beta, g, kappa), eps)
        for _ in range(LH):
            H = _floor(_bmm_h_update(V, W, H, beta, g, kappa), eps)
    elif order == "H":
        for _ in range(LH):
            H = _floor(_bmm_h_update(V, W, H, beta, g, kappa), eps)
        for _ in range(LW):
            W = _floor(_bmm_w_update(V, W, H, beta, g, kappa), eps)
    else:
        raise ValueError(order)
    return W, H


# ---------------------------------------------------------------------------
# Normalisation, stopping rule, driver (Sec. 4.1.2)
# ---------------------------------------------------------------------------

def normalize(W, H):
    """Divide each column of W by its l2 norm and scale the row of H by it."""
    W = W.copy()
    H = H.copy()
    norms = np.sqrt(np.sum(W * W, axis=0))
    nz = norms > 0
    W[:, nz] = W[:, nz] / norms[nz]
    H[nz, :] = H[nz, :] * norms[nz, None]
    return W, H


def run(V, W0, H0, beta: float, method: str = "jmm", iters: int = 100,
        tol: float | None = None, order: str = "W", L: int = 1,
        kappa: float = 0.0, do_normalize: bool = True, gamma_one: bool = False,
        eps: float = 0.0):
    """Outer loop of Algorithm 1 / 2 with the Sec. 4.1.2 stopping rule.

    Runs at most `iters` outer iterations; with `tol`, stops at the first
    iteration where (D_prev - D_cur) / D_cur <= tol. Returns
    (W, H, losses) where losses[i] = D_beta(V + kappa | W_i H_i + kappa) and
    losses[0] is the objective at the initial point.
    """
    W, H = np.array(W0, dtype=np.float64), np.array(H0, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    losses = [D_beta(V + kappa, W @ H + kappa, beta)]
    for _ in range(iters):
        if method == "jmm":
            W, H = jmm_iteration(V, W, H, beta, L=L, order=order, kappa=kappa,
                                 gamma_one=gamma_one, eps=eps)
        elif method == "bmm":
            W, H = bmm_iteration(V, W, H, beta, LW=L, LH=L, order=order,
                                 kappa=kappa, gamma_one=gamma_one, eps=eps)
        else:
            raise ValueError(method)
        if do_normalize:
            W, H = normalize(W, H)
        losses.append(D_beta(V + kappa, W @ H + kappa, beta))
        if tol is not None and (losses[-2] - losses[-1]) / losses[-1] <= tol:
            break
    return W, H, np.array(losses)


# ---------------------------------------------------------------------------
# Gradient and KKT residuals (Sec. 4.1.5)
# ---------------------------------------------------------------------------

def gradients(V, W, H, beta: float, kappa: float = 0.0):
    """Gradient of D_beta(V + kappa | WH + kappa) in W and in H:
    grad_W = [(WH)^(b-2) . (WH - V)] H^T, grad_H = W^T [(WH)^(b-2) . (WH - V)]
    (the terms inside the KKT residuals of Sec. 4.1.5)."""
    WH = W @ H + kappa
    E = WH ** (beta - 2.0) * (WH - (V + kappa))
    return E @ H.T, W.T @ E


def kkt_residuals(V, W, H, beta: float, kappa: float = 0.0):
    """res(W) = ||min{W, grad_W}||_1 / (FK), res(H) = ||min{H, grad_H}||_1 / (KN)."""
    gW, gH = gradients(V, W, H, beta, kappa)
    F, K = W.shape
    N = H.shape[1]
    return (float(np.sum(np.abs(np.minimum(W, gW)))) / (F * K),
            float(np.sum(np.abs(np.minimum(H, gH)))) / (K * N))


# ---------------------------------------------------------------------------
# Sparse count data, beta = 1 (Sec. 4.4 workload; Table 2 row beta = 1)
# ---------------------------------------------------------------------------
# V is given by its nonzeros (rows, cols, vals). Zeros of V contribute
# d_1(0 | y) = y to the objective and nothing to the numerators, because
# A = V / Vt vanishes there and B = Vt^0 = 1 everywhere.

def _sparse_vt(rows, cols, W, H, kappa):
    return np.sum(W[rows, :] * H[:, cols].T, axis=1) + kappa


def _sparse_mul(rows, cols, vals, shape, X_right=None, X_left=None):
    """Sparse-dense products of the COO matrix (rows, cols, vals) of `shape`:
    S @ X_right (X_right is N x K) or X_left^T @ S (X_left is F x K)."""
    import scipy.sparse as sp
    S = sp.coo_matrix((vals, (rows, cols)), shape=shape).tocsr()
    if X_right is not None:
        return np.asarray(S @ X_right)
    return np.asarray((S.T @ X_left).T)


def sparse_kl_objective(rows, cols, vals, W, H, kappa: float = 0.0) -> float:
    """D_1(V | WH) over all F x N entries with V zero off its nonzeros:
    sum_nz [v log(v / vt) - v + vt] + sum over zeros of vt, and the zeros'
    sum is sum_k colsum(W)_k rowsum(H)_k minus the product at the nonzeros.
    With kappa > 0 the zeros have v = kappa and use d_1(kappa | vt)."""
    F, N = W.shape[0], H.shape[1]
    vt = _sparse_vt(rows, cols, W, H, kappa)
    v = vals + kappa
    d_nz = np.sum(beta_divergence(v, vt, 1.0))
    if kappa == 0.0:
        total_product = float(np.sum(W.sum(axis=0) * H.sum(axis=1)))
        return float(d_nz + total_product - np.sum(vt))
    # kappa > 0: zeros contribute d_1(kappa | [WH]_fn + kappa); needs the dense product
    WH = W @ H + kappa
    Vd = np.full((F, N), kappa)
    Vd[rows, cols] = v
    return D_beta(Vd, WH, 1.0)


def sparse_kl_jmm_iteration(rows, cols, vals, Wt, Ht, order: str = "W"):
    """Algorithm 2 at beta = 1, L = 1, kappa = 0 on sparse V.

    beta = 1 gives gamma = 1, chi1(X, Xt) = Xt, chi2(X, Xt) = X (Sec. 3.2), and
    the Table 2 JMM form: W = Wt . (A Ht^T) / (1 H^T), H = Ht . (Wt^T A) / (W^T 1)
    with A = V / (Wt Ht) nonzero only on the support of V.
    """
    F, K = Wt.shape
    N = Ht.shape[1]
    vt = _sparse_vt(rows, cols, Wt, Ht, 0.0)
    a = vals / vt
    AHt = _sparse_mul(rows, cols, a, (F, N), X_right=Ht.T)        # F x K
    WtA = _sparse_mul(rows, cols, a, (F, N), X_left=Wt)            # K x N
    if order == "W":
        W = Wt * AHt / Ht.sum(axis=1)[None, :]                     # chi2(Ht, Ht) = Ht
        H = Ht * WtA / W.sum(axis=0)[:, None]                      # chi2(W, Wt) = W
    else:
        H = Ht * WtA / Wt.sum(axis=0)[:, None]
        W = Wt * AHt / H.sum(axis=1)[None, :]
    return W, H


def sparse_kl_bmm_iteration(rows, cols, vals, W, H, order: str = "W"):
    """Algorithm 1 at beta = 1, L_W = L_H = 1, kappa = 0 on sparse V
    (Table 2 BMM form); the product is recomputed at the nonzeros before the
    second update."""
    F, K = W.shape
    N = H.shape[1]
    if order == "W":
        a = vals / _sparse_vt(rows, cols, W, H, 0.0)
        W = W * _sparse_mul(rows, cols, a, (F, N), X_right=H.T) / H.sum(axis=1)[None, :]
        a = vals / _sparse_vt(rows, cols, W, H, 0.0)
        H = H * _sparse_mul(rows, cols, a, (F, N), X_left=W) / W.sum(axis=0)[:, None]
    else:
        a = vals / _sparse_vt(rows, cols, W, H, 0.0)
        H = H * _sparse_mul(rows, cols, a, (F, N), X_left=W) / W.sum(axis=0)[:, None]
        a = vals / _sparse_vt(rows, cols, W, H, 0.0)
        W = W * _sparse_mul(rows, cols, a, (F, N), X_right=H.T) / H.sum(axis=1)[None, :]
    return W, H


def sparse_kl_gradients(rows, cols, vals, W, H):
    """Gradient of D_1(V | WH) for sparse V: E = 1 - V / WH, so
    grad_W = 1 H^T - A H^T and grad_H = W^T 1 - W^T A with A = V / WH on the support."""
    F, K = W.shape
    N = H.shape[1]
    a = vals / _sparse_vt(rows, cols, W, H, 0.0)
    gW = H.sum(axis=1)[None, :] - _sparse_mul(rows, cols, a, (F, N), X_right=H.T)
    gH = W.sum(axis=0)[:, None] - _sparse_mul(rows, cols, a, (F, N), X_left=W)
    return np.broadcast_to(gW, (F, K)).copy(), np.broadcast_to(gH, (K, N)).copy()


# ---------------------------------------------------------------------------
# Many independent problems (Sec. 4.5 workload shape)
# ---------------------------------------------------------------------------

def batched_run(problems, beta: float, method: str = "jmm", iters: int = 1,
                order: str = "W", do_normalize: bool = True):
    """Runs `run` on each (V, W0, H0) independently; returns a list of
    (W, H, losses). Independent problems share nothing, so a batch is a loop."""
    return [run(V, W0, H0, beta, method=method, iters=iters, order=order,
                do_normalize=do_normalize)
            for (V, W0, H0) in problems]
