"""Gradients of a loss on the label probabilities w.r.t. the edge weights and beta (oracle, FP64).

The paper has no gradients; they differentiate its equations.  Exact path: U_n solves
r(U_n, w) = [(L + gamma D~) U - gamma D~ P]_n = 0 (Eq. rw_eq, normalized form of Sec. II-C with
D~ = D; D~ = I unnormalized), U_s fixed.  With G = d loss / d U_n and the adjoint A lambda = G
(A = L_n + gamma D~_n is symmetric), d loss / d w_e = -lambda-bar^T (d r / d w_e), lambda-bar the
adjoint padded with zeros on the seeds.  For the edge e = (a, b), d L / d w_e = (e_a - e_b)
(e_a - e_b)^T and d D / d w_e = e_a e_a^T + e_b e_b^T, so

  d loss / d w_e = - sum_k [ (lam_a - lam_b)(u_a - u_b)
                             + c gamma (lam_a (u_a - p_a) + lam_b (u_b - p_b)) ],

c = 1 with the normalized Laplacian, 0 otherwise.  d loss / d beta = sum_e (d loss / d w_e)
(d w_e / d beta) with d w_e / d beta from Eq. (W).  The priors depend on the intensities only.

Fast path (``fast_grad``, normalized form only): the loss through the eigenvector solve of
Sec. II-B with Q fixed, the values lambda-hat(w) from Eq. (z_ray) under the current weights, a
fixed m and k damped-Jacobi refinement steps, differentiated in reverse order of the forward
steps (refinement, U = Q_n Lambda_gamma (Q_s^T F_s + gamma Z), the S x S system of Eq. (Fs),
X = B-hat Q_n, Z = Q_n^T P-hat_n, L-hat_s U-hat_s, the Rayleigh values, the coefficients
c_ab = w_ab d_a^{-1/2} d_b^{-1/2}, the scalings d^{+-1/2} and the degrees).  The priors depend on
the intensities only.  ``fd_grad`` gives central differences of any loss of a graph.
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .exact import exact_rw, onehot, split, system
from .graph import edge_dweight_dbeta


def mask_loss(U, truth, seed_idx, label=1):
    """loss = sum over unseeded voxels of (U[x, label] - truth[x])^2 and its gradient."""
    n = split(U.shape[0], seed_idx)
    diff = U[n, label] - truth[n]
    G = np.zeros_like(U)
    G[n, label] = 2.0 * diff
    return float(diff @ diff), G


def exact_grad(g, seed_idx, seed_lab, n_labels, P, gamma, dloss_dU, normalized=True, U=None,
               method="splu", tol=1e-12):
    """Returns (dloss/dw over g.ids order, dloss/dbeta).  The forward and the adjoint system are
    solved by SuperLU (``method="splu"``) or, for graphs too large to factor (3-D volumes), by
    FP64 conjugate gradients to ||r|| <= tol ||b|| per column (``method="cg"``)."""
    if U is None:
        U = exact_rw(g, seed_idx, seed_lab, n_labels, P, gamma, normalized, method=method,
                     tol=tol)
    A, _, n = system(g, seed_idx, seed_lab, n_labels, P, gamma, normalized)
    G = np.asarray(dloss_dU[n])
    if method == "splu":
        lam_n = spla.splu(A.tocsc()).solve(G)
    elif method == "cg":
        lam_n = np.zeros_like(G)
        for k in range(G.shape[1]):
            if not np.any(G[:, k]):
                continue
            x, info = spla.cg(A, G[:, k], rtol=tol, atol=0.0, maxiter=200000)
            if info != 0:
                raise RuntimeError("CG did not converge")
            lam_n[:, k] = x
    else:
        raise ValueError(method)
    lam = np.zeros_like(U)
    lam[n] = lam_n
    a, b = g.a, g.b
    gw = -np.sum((lam[a] - lam[b]) * (U[a] - U[b]), axis=1)
    if normalized and gamma > 0:
        gw -= gamma * np.sum(lam[a] * (U[a] - P[a]) + lam[b] * (U[b] - P[b]), axis=1)
    dwdb = edge_dweight_dbeta(g.J, a, b, g.w, g.form)
    return gw, float(gw @ dwdb)


def fast_forward(g, Q, lam, seed_idx, seed_lab, n_labels, P, gamma, refine_steps=3,
                 omega=0.8):
    """The fast solve (normalized form) with every intermediate kept for ``fast_grad``:
    Eqs. (Fs), (U_lin_comb) with the given values, then damped-Jacobi refinement on the hat
    system (L-hat_n + gamma I) U-hat_n = gamma P-hat_n - B-hat^T U-hat_s."""
    N = g.N
    n = split(N, seed_idx)
    s = np.asarray(seed_idx)
    d = g.d
    sc, sq = 1.0 / np.sqrt(d), np.sqrt(d)
    Cmat = (sp.diags(sc) @ g.W @ sp.diags(sc)).tocsr()     # c_ab = w_ab s_a s_b
    Q = np.asarray(Q, dtype=np.float64)
    lg = 1.0 / (np.asarray(lam, dtype=np.float64) + gamma)
    Qs, Qn = Q[s], Q[n]
    Us = sq[s, None] * onehot(seed_lab, n_labels)
    Css, Csn, Cns, Cnn = Cmat[s][:, s], Cmat[s][:, n], Cmat[n][:, s], Cmat[n][:, n]
    X = -np.asarray(Csn @ Qn)                               # B-hat Q_n, B-hat = -C_sn
    Ph = sq[:, None] * P
    Z = Qn.T @ Ph[n]
    LsUs = Us - np.asarray(Css @ Us)
    rhs = LsUs + gamma * (Us + X @ (lg[:, None] * Z))
    M = np.eye(s.size) - X @ (lg[:, None] * Qs.T)
    Fs = np.linalg.solve(M, rhs)
    Y = Qs.T @ Fs + gamma * Z
    Cm = lg[:, None] * Y
    xs = [Qn @ Cm]
    b = gamma * Ph[n] + np.asarray(Cns @ Us)                # gamma P-hat_n - B-hat^T U-hat_s
    a = omega / (1.0 + gamma)
    for _ in range(refine_steps):
        x = xs[-1]
        xs.append((1.0 - omega) * x + a * np.asarray(Cnn @ x) + a * b)
    U = np.zeros((N, n_labels))
    U[s] = onehot(seed_lab, n_labels)
    U[n] = sc[n, None] * xs[-1]
    return U, dict(n=n, s=s, sc=sc, sq=sq, Cmat=Cmat, lg=lg, Qs=Qs, Qn=Qn, Us=Us, X=X, Ph=Ph,
                   Z=Z, M=M, Fs=Fs, Y=Y, Cm=Cm, xs=xs, b=b, a=a, omega=omega, P=P, Q=Q,
                   gamma=gamma)


def fast_grad(g, Q, seed_idx, seed_lab, n_labels, P, gamma, dloss_dU, refine_steps=3,
              omega=0.8):
    """d loss / d w (over g.ids order) and d loss / d beta through ``fast_forward`` with
    lambda-hat = Rayleigh quotients of Q under g (Eq. z_ray).  Returns (gw, gbeta, U)."""
    from .update import rayleigh_quotients
    Q = np.asarray(Q, dtype=np.float64)
    lam = rayleigh_quotients(Q, g.Lhat)
    U, t = fast_forward(g, Q, lam, seed_idx, seed_lab, n_labels, P, gamma, refine_steps, omega)
    N, n, s = g.N, t["n"], t["s"]
    sc, sq, lg, Qs, Qn = t["sc"], t["sq"], t["lg"], t["Qs"], t["Qn"]
    Cmat, xs, a = t["Cmat"], t["xs"], t["a"]
    ea, eb = g.a, g.b

    def lift(rows, V):
        F = np.zeros((N, V.shape[1]))
        F[rows] = V
        return F

    in_n = np.zeros(N, bool)
    in_n[n] = True
    in_s = ~in_n
    cbar = np.zeros(ea.size)             # d loss / d c_e, both orientations of each edge
    sbar = np.zeros(N)                   # d loss / d s   (s = d^{-1/2})
    sqbar = np.zeros(N)                  # d loss / d sq  (sq = d^{1/2})

    def pair(mask_ab, A_, B_):
        """sum over the entries (a, b) of the selected orientation: A_[a] . B_[b]"""
        out = np.zeros(ea.size)
        out[mask_ab] = np.einsum("ij,ij->i", A_[ea[mask_ab]], B_[eb[mask_ab]])
        return out

    # U_n = s_n x_k
    G = np.asarray(dloss_dU, dtype=np.float64)[n]
    xbar = sc[n, None] * G
    sbar[n] += np.einsum("ij,ij->i", G, xs[-1])
    bbar = np.zeros_like(t["b"])
    Cnn = Cmat[n][:, n]
    for k in range(len(xs) - 1, 0, -1):
        # x_k = (1 - omega) x_{k-1} + a C_nn x_{k-1} + a b
        XB, XT = lift(n, xbar), lift(n, xs[k - 1])
        nn = in_n[ea] & in_n[eb]
        cbar += a * (pair(nn, XB, XT) + pair(nn, XT, XB))
        bbar += a * xbar
        xbar = (1.0 - t["omega"]) * xbar + a * np.asarray(Cnn @ xbar)
    # b = gamma P-hat_n + C_ns U-hat_s
    Phbar = lift(n, t["gamma"] * bbar)
    BB, US = lift(n, bbar), lift(s, t["Us"])
    ns_, sn_ = in_n[ea] & in_s[eb], in_s[ea] & in_n[eb]
    cbar += pair(ns_, BB, US) + pair(sn_, US, BB)
    Usbar = np.asarray(Cmat[s][:, n] @ bbar)
    # x_0 = Q_n Cm,  Cm = lg * Y,  Y = Q_s^T F_s + gamma Z
    Cmbar = Qn.T @ xbar
    Ybar = lg[:, None] * Cmbar
    lgbar = np.einsum("ik,ik->i", Cmbar, t["Y"])
    Fsbar = Qs @ Ybar
    Zbar = t["gamma"] * Ybar
    # F_s = M^{-1} rhs
    rbar = np.linalg.solve(t["M"].T, Fsbar)
    X, Z, Fs = t["X"], t["Z"], t["Fs"]
    # M = I - X diag(lg) Q_s^T, Mbar = -rbar F_s^T
    Xbar = rbar @ (Fs.T @ (Qs * lg[None, :]))
    lgbar += np.einsum("ik,ik->i", X.T @ rbar, Qs.T @ Fs)
    # rhs = L-hat_s U-hat_s + gamma U-hat_s + gamma X (lg Z)
    gam = t["gamma"]
    Usbar += gam * rbar
    Xbar += gam * rbar @ (lg[:, None] * Z).T
    XtR = gam * (X.T @ rbar)
    lgbar += np.einsum("ik,ik->i", XtR, Z)
    Zbar += lg[:, None] * XtR
    # L-hat_s U-hat_s = U-hat_s - C_ss U-hat_s
    Usbar += rbar - np.asarray(Cmat[s][:, s] @ rbar)
    RB = lift(s, rbar)
    ss_ = in_s[ea] & in_s[eb]
    cbar -= pair(ss_, RB, US) + pair(ss_, US, RB)
    # X = -C_sn Q_n
    XBf = lift(s, Xbar)
    cbar -= pair(sn_, XBf, t["Q"]) + pair(ns_, t["Q"], XBf)
    # Z = Q_n^T P-hat_n, P-hat = sq P
    Phbar += lift(n, Qn @ Zbar)
    sqbar += np.einsum("ij,ij->i", Phbar, t["P"])
    # U-hat_s = sq_s onehot
    sqbar[s] += Usbar[np.arange(s.size), np.asarray(seed_lab)]
    # lg = 1 / (lambda-hat + gamma); lambda-hat_i = sum_e w_e (q_ia s_a - q_ib s_b)^2 / |q_i|^2
    lhbar = -lgbar * lg * lg
    qn2 = np.einsum("ij,ij->j", t["Q"], t["Q"])
    coef = lhbar / qn2
    Dq = t["Q"][ea] * sc[ea, None] - t["Q"][eb] * sc[eb, None]          # edges x m
    wbar = (Dq * Dq) @ coef
    tmp = 2.0 * g.w[:, None] * Dq * coef[None, :]
    np.add.at(sbar, ea, np.einsum("em,em->e", tmp, t["Q"][ea]))
    np.add.at(sbar, eb, -np.einsum("em,em->e", tmp, t["Q"][eb]))
    # c_e = w_e s_a s_b
    wbar += cbar * sc[ea] * sc[eb]
    np.add.at(sbar, ea, cbar * g.w * sc[eb])
    np.add.at(sbar, eb, cbar * g.w * sc[ea])
    # s = d^{-1/2}, sq = d^{1/2}, d_a = sum of the weights at a
    dbar = sbar * (-0.5) * g.d ** -1.5 + sqbar * 0.5 * g.d ** -0.5
    wbar += dbar[ea] + dbar[eb]
    dwdb = edge_dweight_dbeta(g.J, ea, eb, g.w, g.form)
    return wbar, float(wbar @ dwdb), U


def fd_grad(loss_of_graph, g, edge_pos=None, h_beta=1e-4, h_rel=1e-4, beta=True):
    """Central differences: d loss / d beta (absolute step h_beta) and d loss / d w_e for the
    edges at positions ``edge_pos`` of g.ids (relative step h_rel * w_e)."""
    from .graph import build_graph
    out = {}
    if beta:
        lp = loss_of_graph(build_graph(g.J, g.dims, g.beta + h_beta, g.form))
        lm = loss_of_graph(build_graph(g.J, g.dims, g.beta - h_beta, g.form))
        out["beta"] = (lp - lm) / (2 * h_beta)
    if edge_pos is not None:
        ge = []
        for p in edge_pos:
            h = h_rel * g.w[p]
            wp = g.w.copy(); wp[p] += h
            wm = g.w.copy(); wm[p] -= h
            ge.append((loss_of_graph(g.with_weights(wp)) - loss_of_graph(g.with_weights(wm)))
                      / (2 * h))
        out["edges"] = np.array(ge)
    return out


__all__ = ["mask_loss", "exact_grad", "fast_forward", "fast_grad", "fd_grad", "onehot"]
