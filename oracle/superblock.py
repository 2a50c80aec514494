"""Superblock Hamiltonian and H·v of the direct n-leg DMRG (oracle; test infrastructure only).

Superblock (paper Fig. 2): block 1 (m1 states, index i1) · block 2 = column
(d states, i2) · block 3 = column (d states, i3) · block 4 (m4 states, i4).

Eq. (dec) splits the Hamiltonian into three parts,

    H = H_l (x) delta_{i3 i4} + H_r (x) delta_{i1 i2} + H_c (x) delta_{i1 i4},

H_l acting on (i1, i2), H_r on (i3, i4), H_c on (i2, i3).  The vector element
of state |i1 i2 i3 i4> sits at 0-based position

    i1 + m1*i2 + m1*d*i4 + m1*d*m4*i3

(the paper's 1-based ((i3-1) m^2 n + (i4-1) m n + (i2-1) m + i1) with n read
as the column dimension d and m1 = m4 = m), and goes to element
(i1 + m1*i2, i4 + m4*i3) of the (m1 d) x (d m4) matrix V: V is the
column-major view of v.  Then H_l v -> H_l V and H_r v -> V H_r^T.  The same
element goes to (i2 + d*i3, i1 + m1*i4) of the d^2 x (m1 m4) matrix V_c and
H_c v -> H_c V_c (paper, text after Eq. (dec)).

Each part is a sum of Kronecker products of a column operator and a block
operator ("terms").  Row/column index order inside H_l is i1 + m1*i2, so a
left term is kron(X_col, Y_block); inside H_r it is i4 + m4*i3, so a right
term is kron(X_col, Y_block); inside H_c it is i2 + d*i3, so a centre term
(a acting on i2, b acting on i3) is kron(b, a).

Fermion signs (the paper is silent): global mode order is block 1, column 2
(legs 0..n-1, spin up then down per site), column 3, block 4; an operator of
subsystem X carries the parities of all subsystems before X.  This gives

    c^dag_{1,e} c_{2,y} = (c^dag_e P_1) (x) c_y     (block first)
    c^dag_{3,y} c_{4,e} = (c^dag_y P_3) (x) c_e
    c^dag_{2,y} c_{3,y} = (c^dag_y P_2) (x) c_y

with P_X the parity of subsystem X and the column c_y carrying its in-column
string.  The spectrum does not depend on this choice; the brute-force ED in
``lattice_ed`` pins it.
"""
from __future__ import annotations

import numpy as np

from .columns import HubbardColumn, SpinColumn


class Superblock:
    """Superblock of a Heisenberg or Hubbard n-leg ladder with given blocks 1 and 4."""

    def __init__(self, model: dict, left: dict, right: dict):
        self.model = model
        self.kind = model["kind"]
        n = int(model["n_legs"])
        self.n_legs = n
        self.left, self.right = left, right
        self.m1, self.m4 = int(left["m"]), int(right["m"])
        if self.kind == "heisenberg":
            col = SpinColumn(n, model["J_rung"], model.get("rung_pbc", False))
        elif self.kind == "hubbard":
            col = HubbardColumn(n, model["t"], model["U"], model.get("rung_pbc", False))
        else:
            raise ValueError(self.kind)
        self.col = col
        self.d = col.d
        self._build_terms()

    # ---- Eq. (dec): the three parts as lists of Kronecker terms ---------------------
    def _build_terms(self):
        col, m1, m4, d = self.col, self.m1, self.m4, self.d
        L = [(1.0, np.eye(d), np.asarray(self.left["H"], float)), (1.0, col.H, np.eye(m1))]
        R = [(1.0, np.eye(d), np.asarray(self.right["H"], float)), (1.0, col.H, np.eye(m4))]
        C = []
        le, re = self.left["edge"], self.right["edge"]
        if self.kind == "heisenberg":
            J = self.model["J_leg"]
            for y in range(self.n_legs):
                if le:
                    sz1, sp1 = np.asarray(le[2 * y]), np.asarray(le[2 * y + 1])
                    L += [(J, col.Sz[y], sz1), (0.5 * J, col.Sm[y], sp1), (0.5 * J, col.Sp[y], sp1.T)]
                if re:
                    sz4, sp4 = np.asarray(re[2 * y]), np.asarray(re[2 * y + 1])
                    R += [(J, col.Sz[y], sz4), (0.5 * J, col.Sp[y], sp4.T), (0.5 * J, col.Sm[y], sp4)]
                C += [(J, col.Sz[y], col.Sz[y]), (0.5 * J, col.Sp[y], col.Sm[y]),
                      (0.5 * J, col.Sm[y], col.Sp[y])]
        else:
            t = self.model["t"]
            P1 = np.diag(np.asarray(self.left["parity"], float))
            P = col.P
            for y in range(self.n_legs):
                for s in range(2):
                    if le:
                        E = np.asarray(le[2 * y + s]) @ P1            # c^dag_{1,e} P_1
                        L += [(-t, col.c[y][s], E), (-t, col.cdag[y][s], E.T)]
                    if re:
                        c4d = np.asarray(re[2 * y + s])               # c^dag_{4,e}
                        R += [(-t, col.cdag[y][s] @ P, c4d.T), (-t, P @ col.c[y][s], c4d)]
                    C += [(-t, col.cdag[y][s] @ P, col.c[y][s]), (-t, P @ col.c[y][s], col.cdag[y][s])]
        self.terms_l, self.terms_r, self.terms_c = L, R, C

    @property
    def n_vec(self) -> int:
        return self.m1 * self.d * self.d * self.m4

    # ---- v <-> 4-index tensor W[i1, i2, i4, i3] --------------------------------------
    def tensor(self, v: np.ndarray) -> np.ndarray:
        return np.asarray(v).reshape((self.m1, self.d, self.m4, self.d), order="F")

    @staticmethod
    def flat(W: np.ndarray) -> np.ndarray:
        return W.reshape(-1, order="F")

    # ---- H·v, 4-index form of Eq. (dec) ----------------------------------------------
    def apply(self, v: np.ndarray) -> np.ndarray:
        """y = H v, each Kronecker term of Eq. (dec) contracted on its own indices."""
        W = self.tensor(v)
        out = np.zeros_like(W)
        for c, X, Y in self.terms_l:      # (X on i2) (Y on i1), identity on i3, i4
            out += c * np.einsum("ia,jb,abkl->ijkl", Y, X, W, optimize=True)
        for c, X, Y in self.terms_r:      # (X on i3) (Y on i4), identity on i1, i2
            out += c * np.einsum("ka,lb,ijab->ijkl", Y, X, W, optimize=True)
        for c, a, b in self.terms_c:      # (a on i2) (b on i3), identity on i1, i4
            out += c * np.einsum("jb,lc,ibkc->ijkl", a, b, W, optimize=True)
        return self.flat(out)

    def apply_slab(self, v: np.ndarray, rows, cols) -> np.ndarray:
        """out[i1 in rows, i2, i4, i3 in cols] of y = H v, the same terms as apply().

        Used to time a bounded sample of a large superblock: H_l terms need only
        the rows ``rows`` of their block operators and the i3 = cols part of v;
        H_r and H_c terms need only the i1 = rows part of v.
        """
        W = self.tensor(v)
        rows, cols = np.asarray(rows), np.asarray(cols)
        Wc = W[:, :, :, cols]
        Wr = W[rows, :, :, :]
        out = np.zeros((len(rows), self.d, self.m4, len(cols)))
        for c, X, Y in self.terms_l:
            out += c * np.einsum("ia,jb,abkl->ijkl", Y[rows, :], X, Wc, optimize=True)
        for c, X, Y in self.terms_r:
            out += c * np.einsum("ka,lb,ijab->ijkl", Y, X[cols, :], Wr, optimize=True)
        for c, a, b in self.terms_c:
            out += c * np.einsum("jb,lc,ibkc->ijkl", a, b[cols, :], Wr, optimize=True)
        return out

    # ---- the paper's matrix forms: H_l V + V H_r^T + H_c V_c ---------------------------
    def H_left(self) -> np.ndarray:
        return sum(c * np.kron(X, Y) for c, X, Y in self.terms_l)

    def H_right(self) -> np.ndarray:
        return sum(c * np.kron(X, Y) for c, X, Y in self.terms_r)

    def H_center(self) -> np.ndarray:
        return sum(c * np.kron(b, a) for c, a, b in self.terms_c)

    def V_of(self, v: np.ndarray) -> np.ndarray:
        return np.asarray(v).reshape((self.m1 * self.d, self.d * self.m4), order="F")

    def Vc_of(self, v: np.ndarray) -> np.ndarray:
        W = self.tensor(v)                                   # [i1, i2, i4, i3]
        return W.transpose(1, 3, 0, 2).reshape((self.d * self.d, self.m1 * self.m4), order="F")

    def v_of_Vc(self, Vc: np.ndarray) -> np.ndarray:
        T = Vc.reshape((self.d, self.d, self.m1, self.m4), order="F")   # [i2, i3, i1, i4]
        return self.flat(T.transpose(2, 0, 3, 1))

    def apply_matrix_form(self, v: np.ndarray) -> np.ndarray:
        """y = H_l V + V H_r^T + H_c V_c, mapped back to vector order (small sizes)."""
        V = self.V_of(v)
        Y = self.H_left() @ V + V @ self.H_right().T
        return Y.reshape(-1, order="F") + self.v_of_Vc(self.H_center() @ self.Vc_of(v))

    def apply_AVB(self, v: np.ndarray) -> np.ndarray:
        """y = H_l V + V H_r^T + sum_k A_k V B_k^T with A_k = a_k (x) I_m1, B_k = b_k (x) I_m4."""
        V = self.V_of(v)
        Y = self.H_left() @ V + V @ self.H_right().T
        for c, a, b in self.terms_c:
            Y += c * np.kron(a, np.eye(self.m1)) @ V @ np.kron(b, np.eye(self.m4)).T
        return Y.reshape(-1, order="F")

    # ---- explicit superblock matrix (small sizes only) ---------------------------------
    def dense(self) -> np.ndarray:
        """Full H with the Kronecker deltas of Eq. (dec) written out, vector index order.

        The flat index is i1 + m1*i2 + m1*d*i4 + m1*d*m4*i3, so the Kronecker
        factor order (most significant first) is (i3, i4, i2, i1).
        """
        d, m1, m4 = self.d, self.m1, self.m4
        I1, I4, Id = np.eye(m1), np.eye(m4), np.eye(d)
        H = np.zeros((self.n_vec, self.n_vec))
        for c, X, Y in self.terms_l:
            H += c * np.kron(np.kron(Id, I4), np.kron(X, Y))
        for c, X, Y in self.terms_r:
            H += c * np.kron(np.kron(X, Y), np.kron(Id, I1))
        for c, a, b in self.terms_c:
            H += c * np.kron(np.kron(b, I4), np.kron(a, I1))
        return H

    # ---- sampled entries of H·v (any size) --------------------------------------------
    def apply_at(self, v: np.ndarray, idx) -> np.ndarray:
        """y[idx] of y = H v, each entry summed straight from Eq. (dec)."""
        W = self.tensor(v)
        m1, d, m4 = self.m1, self.d, self.m4
        out = np.zeros(len(idx))
        for n, f in enumerate(np.asarray(idx, dtype=np.int64)):
            i1 = f % m1
            i2 = (f // m1) % d
            i4 = (f // (m1 * d)) % m4
            i3 = f // (m1 * d * m4)
            s = 0.0
            for c, X, Y in self.terms_l:
                s += c * (Y[i1, :] @ W[:, :, i4, i3] @ X[i2, :])
            for c, X, Y in self.terms_r:
                s += c * (Y[i4, :] @ W[i1, i2, :, :] @ X[i3, :])
            for c, a, b in self.terms_c:
                s += c * (a[i2, :] @ W[i1, :, i4, :] @ b[i3, :])
            out[n] = s
        return out

    # ---- diagonal of H (for the Jacobi preconditioner) --------------------------------
    def diagonal(self) -> np.ndarray:
        m1, d, m4 = self.m1, self.d, self.m4
        D = np.zeros((m1, d, m4, d))
        for c, X, Y in self.terms_l:
            D += c * (np.diag(Y)[:, None] * np.diag(X)[None, :])[:, :, None, None]
        for c, X, Y in self.terms_r:
            D += c * (np.diag(Y)[:, None] * np.diag(X)[None, :])[None, None, :, :]
        for c, a, b in self.terms_c:
            D += c * (np.diag(a)[:, None] * np.diag(b)[None, :])[None, :, None, :]
        return self.flat(D)

    # ---- quantum numbers ----------------------------------------------------------------
    def column_labels(self) -> np.ndarray:
        if self.kind == "heisenberg":
            return self.col.n_up.reshape(-1, 1)
        return np.stack([self.col.n_up, self.col.n_dn], axis=1)

    def sector_mask(self, target) -> np.ndarray:
        """Boolean vector: True where q(i1)+q(i2)+q(i3)+q(i4) equals the target totals."""
        q1 = np.asarray(self.left["qn"], dtype=np.int64)
        q4 = np.asarray(self.right["qn"], dtype=np.int64)
        qc = self.column_labels().astype(np.int64)
        ok = np.ones((self.m1, self.d, self.m4, self.d), dtype=bool)
        for k, tk in enumerate(target):
            tot = (q1[:, k][:, None, None, None] + qc[:, k][None, :, None, None]
                   + q4[:, k][None, None, :, None] + qc[:, k][None, None, None, :])
            ok &= tot == tk
        return self.flat(ok)
