"""Numpy/scipy restatement of the library's Newton-system preconditioner, for
testing the CUDA implementation element by element (test infrastructure; the
preconditioner is a solver choice, not part of the paper's method, so its
reference is a restatement of the same algorithm, not an oracle).

Algorithm (as in the library):
  * scaled system  D J D,  D_ii = |J_ii|^{-1/2} (1 where J_ii = 0);
  * blocks of the unscaled J: A (u-u), B1 (u-p), B2 (p-u), C (p-p);
  * S = C - B2 diag_blocks(A)^{-1} B1 kept on the block sparsity of J, the
    dropped part of every row added to its diagonal; or (fixed stress) S = C
    plus a given lumped term fs on the diagonal of the free pressure rows;
  * z_p = V(S) v_p,  z_u = V(A) (v_u - B1 z_p) (upper order), or
    z_u = V(A) v_u,  z_p = V(S) (v_p - B2 z_u) (lower order); preconditioner
    of the scaled system  z = D^{-1} M^{-1} (D^{-1} v);
  * V-cycle: factor-2 vertex coarsening per axis ((n + 1) // 2 nodes) while
    every axis has more than 2 nodes and the level more than 64 nodes,
    bilinear P (rows of Dirichlet / inactive DOFs zeroed on the finest level),
    Galerkin P^T A P, damped block Jacobi (omega 0.7 in 2D, 0.5 in 3D by
    default, k + k sweeps with k = 1 by default, first sweep from zero),
    exact solve on the coarsest level.
"""
import numpy as np
import scipy.sparse as sps

OMEGA = {2: 0.7, 3: 0.5}   # smoother damping per dimension
PRE, POST = 1, 1


def prolong_1d(nf):
    nc = (nf + 1) // 2
    rows, cols, vals = [], [], []
    for a in range(nf):
        if a % 2 == 0:
            rows.append(a); cols.append(a // 2); vals.append(1.0)
        else:
            rows.append(a); cols.append((a - 1) // 2); vals.append(0.5)
            if (a + 1) // 2 < nc:
                rows.append(a); cols.append((a + 1) // 2); vals.append(0.5)
    return sps.csr_matrix((vals, (rows, cols)), shape=(nf, nc)), nc


def block_inv(A, B):
    n = A.shape[0] // B
    A = A.tocsr()
    out = []
    for a in range(n):
        M = A[a * B:(a + 1) * B, a * B:(a + 1) * B].toarray()
        try:
            inv = np.linalg.inv(M)
            if not np.all(np.isfinite(inv)):
                raise np.linalg.LinAlgError
        except np.linalg.LinAlgError:
            inv = np.eye(B)
        out.append(sps.csr_matrix(inv))
    return sps.block_diag(out, format="csr")


def hierarchy(A, nn, dim, B, free, omega=None, sweeps=None):
    levels = []
    cur = A.tocsr()
    nnc = list(nn)
    first = True
    while True:
        lev = {"A": cur, "Dinv": block_inv(cur, B), "omega": OMEGA[dim] if omega is None else omega,
               "sweeps": (PRE, POST) if sweeps is None else (sweeps, sweeps)}
        levels.append(lev)
        if min(nnc[:dim]) <= 2 or int(np.prod(nnc)) <= 64 or len(levels) >= 15:
            break
        Ps, new = [], []
        for k in range(dim):
            P1, c = prolong_1d(nnc[k])
            Ps.append(P1)
            new.append(c)
        P = Ps[0]
        for k in range(1, dim):
            P = sps.kron(Ps[k], P)          # x index fastest
        P = sps.kron(P, sps.eye(B)).tocsr()
        if first:
            P = (sps.diags(free.astype(float)) @ P).tocsr()
            first = False
        lev["P"] = P
        cur = (P.T @ cur @ P).tocsr()
        nnc = new + list(nnc[dim:])
    return levels


def vcycle(levels, b, l=0):
    A, Dinv, om = levels[l]["A"], levels[l]["Dinv"], levels[l]["omega"]
    if l == len(levels) - 1:
        return np.linalg.solve(A.toarray(), b)
    pre, post = levels[l].get("sweeps", (PRE, POST))
    x = om * (Dinv @ b)
    for _ in range(pre - 1):
        x = x + om * (Dinv @ (b - A @ x))
    P = levels[l]["P"]
    x = x + P @ vcycle(levels, P.T @ (b - A @ x), l + 1)
    for _ in range(post):
        x = x + om * (Dinv @ (b - A @ x))
    return x


class SchurMG:
    """Preconditioner of D J D for the unscaled block-CSR Jacobian J (after
    Dirichlet elimination) with sparsity (row_ptr, col) and fixed-DOF mask."""

    def __init__(self, J, row_ptr, col, fixed, nn, dim, fs=None, lower=True, omega=None, sweeps=None):
        nb = dim + 1
        J = J.tocsr()
        N = J.shape[0]
        nnod = N // nb
        d = np.abs(J.diagonal())
        self.D = np.where(d > 0, 1.0 / np.sqrt(np.where(d > 0, d, 1.0)), 1.0)
        iu = np.array([a * nb + k for a in range(nnod) for k in range(dim)])
        ip = np.arange(nnod) * nb + dim
        self.iu, self.ip = iu, ip
        A = J[iu][:, iu].tocsr()
        self.B1 = J[iu][:, ip].tocsr()
        B2 = J[ip][:, iu].tocsr()
        self.B2 = B2
        self.lower = lower
        C = J[ip][:, ip].tocsr()
        if fs is not None:
            S = (C + sps.diags(np.where(fixed[ip], 0.0, fs))).tocsr()
        else:
            prod = (B2 @ block_inv(A, dim) @ self.B1).tocsr()
            rows = np.repeat(np.arange(nnod), np.diff(row_ptr))
            pat = sps.csr_matrix((np.ones(len(col)), (rows, col)), shape=(nnod, nnod))
            kept = prod.multiply(pat).tocsr()
            lump = np.asarray(prod.sum(axis=1)).ravel() - np.asarray(kept.sum(axis=1)).ravel()
            S = (C - kept - sps.diags(lump)).tocsr()
        self.LA = hierarchy(A, nn, dim, dim, ~fixed[iu], omega, sweeps)
        self.LS = hierarchy(S, nn, dim, 1, ~fixed[ip], omega, sweeps)

    def apply(self, v):
        vv = v / self.D
        if self.lower:
            zu = vcycle(self.LA, vv[self.iu])
            zp = vcycle(self.LS, vv[self.ip] - self.B2 @ zu)
        else:
            zp = vcycle(self.LS, vv[self.ip])
            zu = vcycle(self.LA, vv[self.iu] - self.B1 @ zp)
        z = np.zeros_like(v)
        z[self.iu] = zu
        z[self.ip] = zp
        return z / self.D


def fixed_stress_diag(w, prep):
    """Lumped fixed-stress term at the start of the first step (Delta J = 1,
    J_n = 1): fs_a = sum_p S'_ap V_p / (dt K_p), K = lambda + 2 G / dim, with
    S' the basis renormalised over the point's active support nodes."""
    d = w.dim
    first, count, S, act = prep["first"], prep["count"], prep["S"], prep["active"]
    nnx = [w.ncell[k] + 1 for k in range(d)] + [1, 1]
    lam = w.E * w.nu / ((1 + w.nu) * (1 - 2 * w.nu))
    G = w.E / (2 * (1 + w.nu))
    coef = w.vol / (w.dt * (lam + 2 * G / d))
    out = np.zeros(int(np.prod(nnx[:d])))
    for p in range(w.n):
        cnt = [count[p, k] if k < d else 1 for k in range(3)]
        nodes, vals = [], []
        for o2 in range(cnt[2]):
            for o1 in range(cnt[1]):
                for o0 in range(cnt[0]):
                    o = (o0, o1, o2)
                    c = [first[p, k] + o[k] if k < d else 0 for k in range(3)]
                    a = c[0] + nnx[0] * (c[1] + nnx[1] * c[2])
                    if act[a]:
                        nodes.append(a)
                        vals.append(np.prod([S[p, k, o[k]] for k in range(d)]))
        tot = sum(vals)
        for a, v in zip(nodes, vals):
            out[a] += v / tot * coef[p]
    return out
