"""Factor decomposition of Section 4.1-4.2, in float64 (oracle side).

Every strictly positive pairwise factor exp(w_e(a, b)) is rewritten as a
mixture of product terms with one binary dual variable per dualised table
entry.

Steps, in the paper's order:
  * Section 4.2 (one-hot encoding): with y = [x_s = i] and z = [x_t = j], the
    table entry (i, j) of log-value l contributes the 2x2 factor
    Q(y, z) = exp(l)^(y z), i.e. Q = [[1, 1], [1, e^l]]; entries with l == 0
    ("1-entries") get no dual variable.
  * Lemma 4: if det Q < 0, swap its rows.
  * Lemma 3: left-multiply by diag(1/p12, 1/p21) to make it symmetric.
  * Lemma 2 with Remark 1: factor the symmetric matrix as B~ B~^T with
    cos(phi), sin(phi) from a = p12 / sqrt(p11 p22).
  * Undo the two left-multiplications on B = P-side factor; C = B~.
  * Theorem 2: alpha_1, alpha_2, q, beta_1, beta_2 from B and C.
The result satisfies, for y, z in {0, 1},
    Q(y, z) = exp(alpha_1 y + alpha_2 z) (1 + exp(q + beta_1 y + beta_2 z)) / (1 + exp(q)).

Which scaling of the table is dualised (the paper only says "proportional
to", Section 4.1) is fixed per model by choose_layout:
  * DIAG  when L >= 3 and every off-diagonal log-entry of every edge is exactly
    zero (Potts-type tables): entries (a, a), m = L, no offsets;
  * PIVOT otherwise: w~(i,j) = w(i,j) - w(i,0) - w(0,j) + w(0,0) for i, j >= 1,
    m = (L-1)^2, offsets w(a,0) - w(0,0) to the source, w(0,b) - w(0,0) to the
    destination and the constant w(0,0) to log Z.
Entry index k: PIVOT k = (i-1)(L-1) + (j-1); DIAG k = a.

The closed form (closed_form) is a derived restatement used only as a pin:
with tau = 2 arccosh(exp(|l|/2)),
  l > 0:  q = -tau, beta_1 = beta_2 = tau, alpha_1 = alpha_2 = (l - tau)/2
  l < 0:  q = 0, beta_1 = -tau, beta_2 = tau, alpha_1 = (l + tau)/2, alpha_2 = (l - tau)/2

Parity: pinned by reconstruction of every factor (1e-12), agreement of the
literal pipeline with the closed form (1e-12), strict positivity of B and C,
and the binary-Ising special case (one dual bit with l = 4J).
"""
from __future__ import annotations

import dataclasses

import numpy as np

LAYOUT_PIVOT = 0
LAYOUT_DIAG = 1


# ----------------------------------------------------------------------------- 2x2 steps

def theorem2_params(B, C):
    """Theorem 2: (alpha1, alpha2, q, beta1, beta2) from P = B C^T.

    B, C are [..., 2, 2]; the paper's 1-based B_{r,c} is B[..., r-1, c-1]."""
    B11, B12, B21, B22 = B[..., 0, 0], B[..., 0, 1], B[..., 1, 0], B[..., 1, 1]
    C11, C12, C21, C22 = C[..., 0, 0], C[..., 0, 1], C[..., 1, 0], C[..., 1, 1]
    alpha1 = np.log(B21 / B11)
    alpha2 = np.log(C21 / C11)
    q = np.log(B12 * C12 / (B11 * C11))
    beta1 = np.log(B22 * B11 / (B12 * B21))
    beta2 = np.log(C22 * C11 / (C12 * C21))
    return alpha1, alpha2, q, beta1, beta2


def lemma2_factor(S):
    """Lemma 2 + Remark 1: symmetric S with det >= 0 as B B^T.

    a = s12 / sqrt(s11 s22); cos(phi) = (sqrt(1+a) + sqrt(1-a))/2 and
    sin(phi) = (sqrt(1+a) - sqrt(1-a))/2, the latter evaluated as
    a / (sqrt(1+a) + sqrt(1-a)) (same value, no cancellation)."""
    s11, s12, s22 = S[..., 0, 0], S[..., 0, 1], S[..., 1, 1]
    a = s12 / np.sqrt(s11 * s22)
    sp, sm = np.sqrt(1.0 + a), np.sqrt(1.0 - a)
    cos_phi = 0.5 * (sp + sm)
    sin_phi = a / (sp + sm)
    B = np.empty(S.shape, np.float64)
    B[..., 0, 0] = np.sqrt(s11) * cos_phi
    B[..., 0, 1] = np.sqrt(s11) * sin_phi
    B[..., 1, 0] = np.sqrt(s22) * sin_phi
    B[..., 1, 1] = np.sqrt(s22) * cos_phi
    return B


def factor_2x2(P):
    """Strictly positive factorisation P = B C^T of strictly positive 2x2
    matrices P [..., 2, 2] with det P != 0 (Lemmas 2-4).  Returns (B, C)."""
    P = np.asarray(P, np.float64)
    det = P[..., 0, 0] * P[..., 1, 1] - P[..., 0, 1] * P[..., 1, 0]
    swap = det < 0
    Ps = P.copy()
    Ps[swap] = P[swap][..., ::-1, :]                                   # Lemma 4
    d1 = 1.0 / Ps[..., 0, 1]; d2 = 1.0 / Ps[..., 1, 0]                 # Lemma 3
    S = Ps.copy()
    S[..., 0, :] *= d1[..., None]
    S[..., 1, :] *= d2[..., None]
    S[..., 1, 0] = S[..., 0, 1]          # symmetric by Lemma 3; remove rounding asymmetry
    Bt = lemma2_factor(S)                                               # Lemma 2
    B = Bt.copy()
    B[..., 0, :] /= d1[..., None]
    B[..., 1, :] /= d2[..., None]
    B[swap] = B[swap][..., ::-1, :]
    return B, Bt


def entry_params_literal(ell):
    """Theorem-2 parameters of the one-hot entry factor Q = [[1,1],[1,e^l]] via
    the Section 4.1 pipeline.  ell: float64 array with no zeros."""
    ell = np.asarray(ell, np.float64)
    Q = np.ones(ell.shape + (2, 2), np.float64)
    Q[..., 1, 1] = np.exp(ell)
    B, C = factor_2x2(Q)
    return theorem2_params(B, C), (B, C)


def closed_form(ell):
    """Derived closed form of entry_params_literal (pin only)."""
    ell = np.asarray(ell, np.float64)
    tau = 2.0 * np.arccosh(np.exp(np.abs(ell) / 2.0))
    pos = ell > 0
    q = np.where(pos, -tau, 0.0)
    beta1 = np.where(pos, tau, -tau)
    beta2 = tau.copy()
    alpha1 = np.where(pos, (ell - tau) / 2.0, (ell + tau) / 2.0)
    alpha2 = (ell - tau) / 2.0
    return alpha1, alpha2, q, beta1, beta2


# ----------------------------------------------------------------------------- tables

def choose_layout(n_labels: int, pair: np.ndarray) -> int:
    if n_labels >= 3 and pair.shape[0] > 0:
        off = ~np.eye(n_labels, dtype=bool)
        if not np.any(pair[:, off] != 0):
            return LAYOUT_DIAG
    return LAYOUT_PIVOT


def entry_positions(n_labels: int, layout: int):
    """(i_k, j_k) for every entry slot k of the layout."""
    L = n_labels
    if layout == LAYOUT_DIAG:
        a = np.arange(L)
        return a, a
    i, j = np.meshgrid(np.arange(1, L), np.arange(1, L), indexing="ij")
    return i.ravel(), j.ravel()


def normalise(pair: np.ndarray, layout: int):
    """Split w_e(a,b) = sum_k ell_k [a=i_k][b=j_k] + off_s(a) + off_t(b) + const.

    Returns ell [E][m], off_s [E][L], off_t [E][L], const [E] (float64)."""
    w = np.asarray(pair, np.float64)
    E, L, _ = w.shape
    if layout == LAYOUT_DIAG:
        ell = np.diagonal(w, axis1=1, axis2=2).copy()
        return ell, np.zeros((E, L)), np.zeros((E, L)), np.zeros(E)
    piv = w - w[:, :, :1] - w[:, :1, :] + w[:, :1, :1]
    ell = piv[:, 1:, 1:].reshape(E, (L - 1) * (L - 1))
    off_s = w[:, :, 0] - w[:, :1, 0]
    off_t = w[:, 0, :] - w[:, 0, :1]
    return ell, off_s, off_t, w[:, 0, 0].copy()


@dataclasses.dataclass
class Decomposition:
    layout: int
    n_labels: int
    i_pos: np.ndarray      # [m] row label of entry k
    j_pos: np.ndarray      # [m] column label of entry k
    ell: np.ndarray        # [E][m] dualised log-entries (0 = no dual variable)
    active: np.ndarray     # [E][m] bool, ell != 0
    alpha1: np.ndarray     # [E][m] Theorem-2 parameters (0 where inactive)
    alpha2: np.ndarray
    q: np.ndarray
    beta1: np.ndarray
    beta2: np.ndarray
    utilde: np.ndarray     # [N][L] unaries with offsets and alpha terms folded in
    log_const: float       # log p~(x) = log sum_theta p~(x, theta) + log_const
    src: np.ndarray
    dst: np.ndarray

    @property
    def n_entries(self) -> int:
        return int(self.i_pos.shape[0])


def decompose(model, layout=None) -> Decomposition:
    """Decompose every pairwise factor of the model (Sections 4.1-4.2, Theorem 1)."""
    L = model.n_labels
    if layout is None:
        layout = choose_layout(L, model.pair)
    ell, off_s, off_t, const = normalise(model.pair, layout)
    i_pos, j_pos = entry_positions(L, layout)
    active = ell != 0
    E, m = ell.shape
    a1 = np.zeros((E, m)); a2 = np.zeros((E, m)); q = np.zeros((E, m))
    b1 = np.zeros((E, m)); b2 = np.zeros((E, m))
    if np.any(active):
        (pa1, pa2, pq, pb1, pb2), _ = entry_params_literal(ell[active])
        a1[active], a2[active], q[active], b1[active], b2[active] = pa1, pa2, pq, pb1, pb2
    N = model.n_vars
    ut = np.asarray(model.unary, np.float64).copy()
    # fold offsets (normalisation) and alpha terms (h(x) of Theorem 2) into unaries
    fold_s = off_s.copy(); fold_t = off_t.copy()
    np.add.at(fold_s, (np.arange(E)[:, None], np.broadcast_to(i_pos, (E, m))), a1)
    np.add.at(fold_t, (np.arange(E)[:, None], np.broadcast_to(j_pos, (E, m))), a2)
    np.add.at(ut, model.src.astype(np.int64), fold_s)
    np.add.at(ut, model.dst.astype(np.int64), fold_t)
    # exp(l y z) = e^{a1 y + a2 z} (1 + e^{q + b1 y + b2 z}) / (1 + e^q)
    log_const = float(const.sum() - np.logaddexp(0.0, q[active]).sum())
    return Decomposition(layout, L, i_pos, j_pos, ell, active, a1, a2, q, b1, b2, ut, log_const,
                         model.src.astype(np.int64), model.dst.astype(np.int64))


def fold_vectors(model, dec: Decomposition):
    """Per-edge unary folds (offsets + alpha terms): fold_s [E][L], fold_t [E][L].
    Used by the blocked sampler to take exact tree edges out of the folded unaries."""
    L = model.n_labels
    _, off_s, off_t, _ = normalise(model.pair, dec.layout)
    E, m = dec.ell.shape
    fold_s = off_s.copy(); fold_t = off_t.copy()
    np.add.at(fold_s, (np.arange(E)[:, None], np.broadcast_to(dec.i_pos, (E, m))), dec.alpha1)
    np.add.at(fold_t, (np.arange(E)[:, None], np.broadcast_to(dec.j_pos, (E, m))), dec.alpha2)
    return fold_s, fold_t
