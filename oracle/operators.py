"""Oracle operators: A, Y, L, U and the block eigenvalues, from their definitions (FP64).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.linalg import toeplitz


def _axes(prob):
    return list(prob.m), list(prob.h)


def laplacian_1d(m: int, h: float) -> sp.csr_matrix:
    """L = -Delta_h in 1-D: the central-difference Dirichlet Laplacian, tridiag(-1, 2, -1)/h^2.

    Sec. 5.2 (central differences on a uniform grid, zero boundary values; Delta_h is symmetric
    negative definite, so L is SPD).
    """
    e = np.ones(m)
    return sp.diags([-e[:-1], 2.0 * e, -e[:-1]], [-1, 0, 1], format="csr") / (h * h)


def laplacian_variable(prob) -> sp.csr_matrix:
    """L_a = -Delta_{a,h}: the central-difference discretisation of -div(a grad) (Sec. 5.2, the
    paper's Delta_{a,h}; Example heateqvarcoeff), zero Dirichlet values, x fastest.

    Along axis ax, point c of a line couples to c-1 and c+1 through the coefficient at the faces
    between them: (L_a u)_c = [a_{c-1/2} (u_c - u_{c-1}) + a_{c+1/2} (u_c - u_{c+1})] / h^2, with
    u = 0 outside.  prob.meta["faces"][ax] holds a at the faces along ax as an array of shape
    (m_z, m_y, m_x) with that axis one longer (face f sits before point f; face m_ax after the last
    point).  Written entry by entry from that formula; the result is symmetric.
    """
    ms, hs = _axes(prob)
    M = int(np.prod(ms))
    shape = tuple(reversed(ms))                       # ([z], [y], x): x is the last array axis
    idx = np.arange(M).reshape(shape)
    rows, cols, vals = [], [], []
    for ax in range(prob.d):
        arr_axis = len(shape) - 1 - ax
        fa = np.asarray(prob.meta["faces"][ax], dtype=np.float64)
        lo = np.take(fa, range(0, ms[ax]), axis=arr_axis)          # a_{c-1/2}
        hi = np.take(fa, range(1, ms[ax] + 1), axis=arr_axis)      # a_{c+1/2}
        h2 = hs[ax] ** 2
        rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append(((lo + hi) / h2).ravel())
        if ms[ax] > 1:
            a_ = np.take(idx, range(0, ms[ax] - 1), axis=arr_axis)
            b_ = np.take(idx, range(1, ms[ax]), axis=arr_axis)
            w = -np.take(hi, range(0, ms[ax] - 1), axis=arr_axis) / h2   # face between a_ and b_
            rows += [a_.ravel(), b_.ravel()]
            cols += [b_.ravel(), a_.ravel()]
            vals += [w.ravel(), w.ravel()]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(M, M))


def dense_eigh(prob):
    """K = U diag(mu) U^T for a problem with a dense symmetric operator prob.meta["K"] (the
    commuting-blocks case of Sec. 3: A_(k) = a_k I + b_k K share the eigenvectors of K); numpy's
    symmetric eigensolver as the step, cached on the problem."""
    c = prob.meta.get("_eigh")
    if c is None:
        c = np.linalg.eigh(np.asarray(prob.meta["K"], dtype=np.float64))
        prob.meta["_eigh"] = c
    return c


def blocks_of(prob):
    """The blocks A_(k), k = 0..N-1, as an (N, M, M) array when the problem gives them as dense
    symmetric matrices (prob.meta["blocks"]: commuting blocks in general, Assumption 1 (i)),
    else None."""
    B = prob.meta.get("blocks")
    return None if B is None else np.asarray(B, dtype=np.float64)


def commuting_eigh(prob):
    """Common orthonormal eigenvectors U of commuting symmetric blocks (Assumption 1 (i), Sec. 3):
    the eigenvectors of one generic combination S = sum_k r_k A_(k) (numpy's symmetric
    eigensolver as the step).  Commuting symmetric matrices are simultaneously diagonalisable,
    and when S has simple eigenvalues its eigenvectors diagonalise every A_(k).  The weights r_k
    are fixed draws from default_rng(20230717).  Cached on the problem."""
    U = prob.meta.get("_ceigh")
    if U is None:
        B = blocks_of(prob)
        r = np.random.default_rng(20230717).standard_normal(B.shape[0])
        S = np.tensordot(r, B, axes=(0, 0))
        U = np.linalg.eigh(0.5 * (S + S.T))[1]
        prob.meta["_ceigh"] = U
    return U


def laplacian(prob) -> sp.csr_matrix:
    """L = -Delta_h on the tensor grid, lexicographic order with x fastest (Sec. 5.2); L_a when
    the problem carries a variable coefficient (prob.meta["faces"], see laplacian_variable); the
    dense symmetric K when it carries one (prob.meta["K"]).

    The d-dimensional operator is the Kronecker sum of the 1-D ones; axis 0 (x) is the fastest.
    """
    if prob.meta.get("K") is not None:
        return sp.csr_matrix(np.asarray(prob.meta["K"], dtype=np.float64))
    if prob.meta.get("faces") is not None:
        return laplacian_variable(prob)
    ms, hs = _axes(prob)
    M = int(np.prod(ms))
    L = sp.csr_matrix((M, M))
    for ax in range(prob.d):
        inner = int(np.prod(ms[:ax]))            # axes faster than this one
        outer = int(np.prod(ms[ax + 1:]))        # axes slower than this one
        term = sp.kron(sp.identity(outer), sp.kron(laplacian_1d(ms[ax], hs[ax]), sp.identity(inner)))
        L = L + term
    return L.tocsr()


def dst1_matrix(m: int) -> np.ndarray:
    """Normalised DST-I matrix S[j, k] = sqrt(2/(m+1)) sin(pi (j+1)(k+1)/(m+1)).

    It is the orthogonal U that diagonalises every block for the paper's examples (Sec. 5.1: the
    blocks are diagonalised by the discrete sine transform).  S is symmetric and S @ S = I.
    """
    j = np.arange(1, m + 1)
    return np.sqrt(2.0 / (m + 1)) * np.sin(np.pi * np.outer(j, j) / (m + 1))


def laplacian_eigenvalues(prob) -> np.ndarray:
    """Eigenvalues mu_i of L in the order of U's columns (lexicographic, x fastest).

    Per axis the 1-D eigenvalue of column k is (4/h^2) sin^2(pi (k+1) / (2 (m+1))) (textbook);
    the d-dimensional ones are their sums over the axes.
    """
    if prob.meta.get("K") is not None:
        return dense_eigh(prob)[0]
    ms, hs = _axes(prob)
    mu = np.zeros(1)
    for ax in range(prob.d):            # build with x fastest: later axes are slower
        k = np.arange(1, ms[ax] + 1)
        mu1 = 4.0 / hs[ax] ** 2 * np.sin(np.pi * k / (2.0 * (ms[ax] + 1))) ** 2
        mu = (mu1[:, None] + mu[None, :]).reshape(-1)
    return mu


def apply_U(prob, V: np.ndarray, transpose: bool = False) -> np.ndarray:
    """Apply I_N (x) U (or (I_N (x) U)^T) to a time-major array V of shape (N, M): the DST-I along
    every spatial axis.

    U = S_z (x) S_y (x) S_x (x fastest) is symmetric and orthogonal, so U^T = U there.  With a
    dense operator K, U holds the eigenvectors of K as columns (dense_eigh) and the two differ.
    Used for Steps 1 (U^T) and 3 (U) of the preconditioner solve (Sec. 5.1).
    """
    if prob.meta.get("K") is not None or prob.meta.get("blocks") is not None:
        U = dense_eigh(prob)[1] if prob.meta.get("K") is not None else commuting_eigh(prob)
        X = np.asarray(V, dtype=np.float64)
        return X @ U if transpose else X @ U.T        # rows are time slices
    ms = list(prob.m)
    N = V.shape[0]
    X = V.reshape((N,) + tuple(reversed(ms)))        # (N, [z], [y], x)
    for ax in range(prob.d):
        S = dst1_matrix(ms[ax])
        arr_axis = X.ndim - 1 - ax                    # x is the last array axis
        X = np.moveaxis(np.tensordot(X, S, axes=([arr_axis], [0])), -1, arr_axis)
    return X.reshape(N, -1)


def block_eigenvalues(prob) -> np.ndarray:
    """lambda_i^(k) = a_k + b_k mu_i, the eigenvalues of A_(k) = U Lambda_k U^T (Sec. 3); for
    general commuting blocks (prob.meta["blocks"]) u_i^T A_(k) u_i with U = commuting_eigh.

    Returns an (N, M) array: row k holds the diagonal of Lambda_k.  For a variable-coefficient
    problem these are the eigenvalues of the mean-coefficient blocks a_k I + abar b_k L (eq.
    meancoeffheateqtsmat, abar = prob.meta["abar"]), from which the preconditioner is built.
    """
    B = blocks_of(prob)
    if B is not None:
        # general commuting blocks: lambda_i^(k) = u_i^T A_(k) u_i in the common eigenbasis
        lam = prob.meta.get("_clam")
        if lam is None:
            U = commuting_eigh(prob)
            lam = np.stack([np.sum(U * (B[k] @ U), axis=0) for k in range(B.shape[0])])
            prob.meta["_clam"] = lam
        return lam
    mu = laplacian_eigenvalues(prob)
    b = prob.b * float(prob.meta.get("abar", 1.0)) if prob.meta.get("faces") is not None else prob.b
    return prob.a[:, None] + b[:, None] * mu[None, :]


def assumption_margin(prob) -> float:
    """c0 = min_i (lambda_i^(0) - sum_{j>=1} |lambda_i^(j)|) (Proposition after Lemma 3.1).

    Assumption 1(ii) holds iff this is positive.  Evaluated over every mode.
    """
    lam = block_eigenvalues(prob)
    return float(np.min(lam[0] - np.abs(lam[1:]).sum(axis=0)))


def bltt_matvec(prob, z: np.ndarray, flip: bool = False) -> np.ndarray:
    """y = A z (or Y A z when flip), A the BLTT matrix of eq. amatdef, computed directly.

    Block row n of A z is sum_{k=0}^{n} A_(k) z_{n-k} = sum_k a_k z_{n-k} + L sum_k b_k z_{n-k}
    (or, for general blocks given as matrices, the block sum itself).
    With Z the (N, M) time-major array, the two time sums are the lower-triangular Toeplitz
    products T_a Z and T_b Z (O(N^2 M), a library matmul as the step), and L acts per time slice.
    Y = Y_N (x) I_M reverses the order of the time blocks (Sec. 2).
    """
    N, M = prob.N, prob.M
    Z = np.asarray(z, dtype=np.float64).reshape(N, M)
    B = blocks_of(prob)
    if B is not None:
        # general blocks: block row n is sum_{k<=n} A_(k) z_{n-k}, one matrix product per k
        Yv = np.zeros((N, M))
        for k in range(N):
            Yv[k:] += Z[:N - k] @ B[k].T
        if flip:
            Yv = Yv[::-1]
        return np.ascontiguousarray(Yv).reshape(-1)
    Ta = toeplitz(prob.a, np.zeros(N))
    Yv = Ta @ Z
    if np.any(prob.b != 0):
        Tb = toeplitz(prob.b, np.zeros(N))
        W = Tb @ Z
        L = laplacian(prob)
        Yv = Yv + (L @ W.T).T
    if flip:
        Yv = Yv[::-1]
    return np.ascontiguousarray(Yv).reshape(-1)


def bltt_matvec_entry(prob, z: np.ndarray, n: int, i: int, flip: bool = False) -> float:
    """One entry of A z (or Y A z): block row n, spatial index i, by the block sum itself.

    Used for sampled checks at sizes where the full product is too slow.
    """
    N, M = prob.N, prob.M
    Z = np.asarray(z).reshape(N, M)
    row = N - 1 - n if flip else n
    B = blocks_of(prob)
    if B is not None:
        return float(sum(B[k][i] @ Z[row - k] for k in range(row + 1)))
    ms = list(prob.m)
    # neighbours of i in the Laplacian stencil
    coords = []
    r = i
    for ax in range(prob.d):
        coords.append(r % ms[ax])
        r //= ms[ax]
    acc = 0.0
    for k in range(row + 1):
        zk = Z[row - k]
        if prob.a[k] != 0.0:
            acc += prob.a[k] * zk[i]
        if prob.b[k] != 0.0 and prob.meta.get("K") is not None:
            acc += prob.b[k] * float(np.asarray(prob.meta["K"])[i] @ zk)
        elif prob.b[k] != 0.0:
            lz = 0.0
            stride = 1
            faces = prob.meta.get("faces")
            for ax in range(prob.d):
                h2 = prob.h[ax] ** 2
                if faces is None:
                    alo = ahi = 1.0
                else:
                    fa = np.asarray(faces[ax])
                    pos = list(reversed(coords))              # ([z], [y], x) array index
                    p_lo = list(pos)
                    p_hi = list(pos)
                    p_hi[len(pos) - 1 - ax] += 1
                    alo, ahi = fa[tuple(p_lo)], fa[tuple(p_hi)]
                lz += (alo + ahi) * zk[i] / h2
                if coords[ax] > 0:
                    lz -= alo * zk[i - stride] / h2
                if coords[ax] < ms[ax] - 1:
                    lz -= ahi * zk[i + stride] / h2
                stride *= ms[ax]
            acc += prob.b[k] * lz
    return acc


def assemble_A(prob) -> np.ndarray:
    """Dense A of eq. amatdef: block (p, q) is A_(p-q) for p >= q, zero above (tiny sizes only)."""
    N, M = prob.N, prob.M
    A = np.zeros((N * M, N * M))
    for p in range(N):
        for q in range(p + 1):
            A[p * M:(p + 1) * M, q * M:(q + 1) * M] = block_matrix(prob, p - q)
    return A


def block_matrix(prob, k: int) -> np.ndarray:
    """A_(k) as a dense M x M matrix: a_k I + b_k L, or the given block (eq. amatdef)."""
    B = blocks_of(prob)
    if B is not None:
        return B[k]
    return prob.a[k] * np.eye(prob.M) + prob.b[k] * laplacian(prob).toarray()


def assemble_Y(N: int, M: int) -> np.ndarray:
    """Dense Y = Y_N (x) I_M, Y_N the anti-identity (Sec. 2)."""
    return np.kron(np.fliplr(np.eye(N)), np.eye(M))


def assemble_C_alpha(prob, alpha: float) -> np.ndarray:
    """Dense block alpha-circulant C_alpha = I_N (x) A_(0) + sum_k H_alpha^(k) (x) A_(k) (eq. tensordef2calpha).

    H_alpha^(k) = [[0, alpha I_k], [I_{N-k}, 0]] (Sec. 3).
    """
    N, M = prob.N, prob.M
    C = np.kron(np.eye(N), block_matrix(prob, 0))
    for k in range(1, N):
        H = np.zeros((N, N))
        H[:k, N - k:] = alpha * np.eye(k)
        H[k:, :N - k] = np.eye(N - k)
        C += np.kron(H, block_matrix(prob, k))
    return C
