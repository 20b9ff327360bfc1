"""Plain, slow FP64 CPU oracle for C4v-symmetric CTMRG and QR-CTMRG.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import or run this module.  The CUDA
library never calls it and shares no code with it.

Every function follows the paper (Zhang, Yang, Corboz, "Accelerating
two-dimensional tensor network contractions using QR-decompositions",
arXiv 2505.00494) and names the passage it restates.  All arithmetic is
written so that it stays analytic when the inputs are complex (no ``conj``,
no ``abs`` on the data path, norms are ``sqrt(sum(x*x))``); this lets a
complex-step derivative ``Im E(A + i h v) / h`` pass through the QR path.

Index conventions (a reading; the paper's figures are not available):

* ``A[s,u,l,d,r]``: physical ``s < d``, virtual up/left/down/right ``< D``
  (iPEPS paragraph, Fig. 1(a)).
* ``a[U,L,Dn,R]`` with ``U = u*D + u'`` (ket-major), ``a = sum_s A (x) A``
  (Fig. 1(b)).
* Corner ``C[alpha,beta]`` (chi x chi), edge ``T[alpha,k,beta]``
  (chi x D^2 x chi); the same C and T stand for all four corners and edges
  (Standard CTMRG paragraph, C4v case).
* Enlarged corner (Fig. 1(d)):
  ``Ct[(b,l),(r,j)] = sum C[g,h] T[h,i,r] T[g,k,b] a[i,k,l,j]``.
* Reduced corner (Fig. 1(e)): ``ct[(g,i),r] = sum_h C[g,h] T[h,i,r]``,
  a (chi D^2) x chi matrix of rank <= chi.

Parity pins for every function live in ``tests/test_oracle_*.py``.  The
unrolled and fixed-point gradients are pinned by complex-step derivatives of
this same module, by central finite differences and by the invariants
<g, A> = 0 and sym(g) = g.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# C4v symmetry (iPEPS paragraph and its footnote on n(D))
# ---------------------------------------------------------------------------

# The 8 elements of C4v acting on the virtual legs (u,l,d,r) of A: four
# rotations (cyclic shifts) and four reflections (reversed cycles).
C4V_PERMS = [
    (0, 1, 2, 3), (1, 2, 3, 0), (2, 3, 0, 1), (3, 0, 1, 2),
    (0, 3, 2, 1), (1, 0, 3, 2), (2, 1, 0, 3), (3, 2, 1, 0),
]


def c4v_sym(X):
    """Projector onto C4v-invariant rank-5 tensors: mean over the 8 group elements."""
    out = np.zeros_like(X)
    for p in C4V_PERMS:
        out = out + np.transpose(X, (0,) + tuple(1 + q for q in p))
    return out / 8.0


def n_params(d: int, D: int) -> float:
    """Number of C4v variational parameters (footnote in the iPEPS paragraph)."""
    return d / 8.0 * (D ** 4 + 2 * D ** 3 + 3 * D ** 2 + 2 * D)


def fro_norm(X):
    """Analytic Frobenius norm sqrt(sum x^2) (no conjugation)."""
    return np.sqrt(np.sum(X * X))


def normalized_input(X):
    """A = sym(X) / ||sym(X)||, the input recipe applied to a raw draw."""
    S = c4v_sym(np.asarray(X))
    return S / fro_norm(S)


# ---------------------------------------------------------------------------
# Double layer and boundary initialisation (Fig. 1(b); footnote on the
# initial boundary in the Standard CTMRG paragraph)
# ---------------------------------------------------------------------------

def double_layer(A):
    """a[(u u'),(l l'),(d d'),(r r')] = sum_s A[s,u,l,d,r] A[s,u',l',d',r']."""
    d, D = A.shape[0], A.shape[1]
    a = np.einsum("suldr,sULDR->uUlLdDrR", A, A)
    return a.reshape(D * D, D * D, D * D, D * D)


def double_layer_open(A):
    """aO[s,t,U,L,Dn,R] = A[s,u,l,d,r] A[t,u',l',d',r']: physical legs left open."""
    d, D = A.shape[0], A.shape[1]
    aO = np.einsum("suldr,tULDR->stuUlLdDrR", A, A)
    return aO.reshape(d, d, D * D, D * D, D * D, D * D)


def init_env(A, fixed_phys=None):
    """Boundary tensors from the bulk: contract ket and bra legs that point out
    of the system (footnote to the Standard CTMRG paragraph).

    Corner (top-left): up and left legs traced, open legs down and right:
        C0[(d d'),(r r')] = sum_{s,u,l} A[s,u,l,d,r] A[s,u,l,d',r'].
    Edge (left column): left leg traced, open legs up, right (inner), down:
        T0[(u u'),(r r'),(d d')] = sum_{s,l} A[s,u,l,d,r] A[s,u',l,d',r'].
    ``fixed_phys`` restricts the physical sum to one index (a fixed boundary
    spin, used for the symmetry-broken classical Ising test).
    """
    D = A.shape[1]
    As = A if fixed_phys is None else A[fixed_phys:fixed_phys + 1]
    C0 = np.einsum("suldr,sulDR->dDrR", As, As).reshape(D * D, D * D)
    T0 = np.einsum("suldr,sUlDR->uUrRdD", As, As).reshape(D * D, D * D, D * D)
    return sym_norm(C0, T0)


def sym_norm(C, T):
    """Impose the reflection symmetry of corner and edge and normalise
    (the paper leaves this step implicit; reading: C <- (C + C^T)/2,
    T[a,k,b] <- (T[a,k,b] + T[b,k,a])/2, each divided by its Frobenius norm).
    """
    C = 0.5 * (C + C.T)
    T = 0.5 * (T + np.transpose(T, (2, 1, 0)))
    return C / fro_norm(C), T / fro_norm(T)


# ---------------------------------------------------------------------------
# Standard C4v CTMRG step (Standard CTMRG paragraph, Fig. 1(c,d))
# ---------------------------------------------------------------------------

def enlarged_corner(C, T, a):
    """Ct[(b,l),(r,j)] = sum_{g,h,i,k} C[g,h] T[h,i,r] T[g,k,b] a[i,k,l,j]
    (contracted pairwise: C T, then the second T, then a)."""
    chi, D2 = T.shape[0], T.shape[1]
    ct = np.tensordot(C, T, axes=([1], [0]))               # [g,i,r]
    X = np.tensordot(ct, T, axes=([0], [0]))               # [i,r,k,b]
    Ct = np.tensordot(X, a, axes=([0, 2], [0, 1]))         # [r,b,l,j]
    return np.transpose(Ct, (1, 2, 0, 3)).reshape(chi * D2, chi * D2)


def renormalize_edge(P, T, a):
    """T'[m,j,n] = sum P[(a,u),m] T[a,k,b] a[u,k,d,j] P[(b,d),n] for an
    isometry P of shape (chi*D2, chi') (U in Fig. 1(d), Q in Fig. 1(e));
    contracted pairwise in the order written."""
    chi, D2 = T.shape[0], T.shape[1]
    P3 = P.reshape(chi, D2, P.shape[1])
    X1 = np.tensordot(P3, T, axes=([0], [0]))              # [u,m,k,b]
    X2 = np.tensordot(X1, a, axes=([0, 2], [0, 1]))        # [m,b,d,j]
    return np.tensordot(X2, P3, axes=([1, 2], [0, 1])).transpose(0, 1, 2)  # [m,j,n]


def eigen_step(C, T, a, chi_target):
    """One standard step: diagonalise the enlarged corner, keep the chi
    eigenvectors of largest |eigenvalue| (ties broken by index), project."""
    Ct = enlarged_corner(C, T, a)
    Ct = 0.5 * (Ct + Ct.T)
    w, V = np.linalg.eigh(Ct)
    n = w.shape[0]
    order = np.lexsort((np.arange(n), -np.abs(w)))
    chi_new = min(chi_target, n)
    U = V[:, order[:chi_new]]
    C_new = U.T @ Ct @ U
    T_new = renormalize_edge(U, T, a)
    return sym_norm(C_new, T_new)


# ---------------------------------------------------------------------------
# Householder QR (QR-CTMRG paragraph: unpivoted QR of the reduced corner)
# ---------------------------------------------------------------------------

def _sign_re(x):
    return 1.0 if np.real(x) >= 0 else -1.0


def householder_qr(M):
    """Thin unpivoted Householder QR, M = Q R with Q^T Q = I and diag(R) >= 0.

    Column j: x = R[j:, j]; the reflector H = I - tau v v^T with
    v = x + sign(x_0) ||x|| e_1 maps x to -sign(x_0) ||x|| e_1.  A zero x
    gives H = I.  At the end the signs of R's rows and Q's columns are flipped
    so that diag(R) >= 0 (sign reading for the unpivoted QR).  Q is formed by
    applying the reflectors in reverse order to the first n columns of I.
    """
    M = np.array(M, copy=True)
    m, n = M.shape
    R = M.copy()
    vs, taus = [], []
    for j in range(n):
        x = R[j:, j].copy()
        if np.all(x == 0):
            vs.append(None)
            taus.append(0.0)
            continue
        nx = np.sqrt(np.sum(x * x))
        s = _sign_re(x[0])
        v = x.copy()
        v[0] = x[0] + s * nx
        tau = 2.0 / np.sum(v * v)
        w = v @ R[j:, j:]
        R[j:, j:] = R[j:, j:] - tau * np.outer(v, w)
        R[j + 1:, j] = 0.0
        vs.append(v)
        taus.append(tau)
    R = np.triu(R[:n, :])
    Q = np.zeros((m, n), dtype=R.dtype)
    Q[np.arange(n), np.arange(n)] = 1.0
    for j in reversed(range(n)):
        v = vs[j]
        if v is None:
            continue
        w = v @ Q[j:, :]
        Q[j:, :] = Q[j:, :] - taus[j] * np.outer(v, w)
    sgn = np.array([_sign_re(R[j, j]) for j in range(n)])
    Q = Q * sgn[None, :]
    R = R * sgn[:, None]
    return Q, R


# ---------------------------------------------------------------------------
# QR-CTMRG step (QR-CTMRG paragraph, Fig. 1(e,f))
# ---------------------------------------------------------------------------

def reduced_corner(C, T):
    """ct[(g,i),r] = sum_h C[g,h] T[h,i,r]: the corner with one row fewer."""
    chi, D2 = T.shape[0], T.shape[1]
    return np.einsum("gh,hir->gir", C, T).reshape(chi * D2, chi)


def absorb_split(X1, A):
    """Double-layer absorption done ket layer then bra layer (no explicit a):
    X2[m,b,d,j] = sum X1[u,m,k,b] a[u,k,d,j] with
    a[u,k,d,j] = sum_s A[s,uk,kk,dk,jk] A[s,ub,kb,db,jb]."""
    D = A.shape[1]
    D2, chi = X1.shape[0], X1.shape[1]
    X = X1.reshape(D, D, chi, D, D, chi)           # [uk,ub,m,kk,kb,b]
    Z = np.tensordot(X, A, axes=([0, 3], [1, 2]))  # ket: [ub,m,kb,b,s,dk,jk]
    X2 = np.tensordot(Z, A, axes=([4, 0, 2], [0, 1, 2]))  # bra: [m,b,dk,jk,db,jb]
    X2 = np.transpose(X2, (0, 1, 2, 4, 3, 5))      # [m,b,dk,db,jk,jb]
    return X2.reshape(chi, chi, D2, D2)            # [m,b,(dk db),(jk jb)]


def qr_step_parts(C, T, A, layers="double"):
    """All intermediates of one QR-CTMRG step (QR-CTMRG paragraph).

    1. ct = C T (Fig. 1(e)), 2. ct = Q R, 3. T' with Q in place of U,
    4. C' from T', R, Q (Fig. 1(f)):
       C'[n,p] = sum_{m,g,j} T'[m,j,n] R[m,g] Q[(g,j),p],
       which equals Q^T Ct Q exactly because Ct = sum_m Y_m R[m,:] after
       substituting ct = Q R into the enlarged corner.
    5. sym_norm.
    """
    chi, D2 = T.shape[0], T.shape[1]
    ct = reduced_corner(C, T)
    Q, R = householder_qr(ct)
    Q3 = Q.reshape(chi, D2, chi)
    if layers in ("double", "network"):
        a = A if layers == "network" else double_layer(A)
        T_raw = renormalize_edge(Q, T, a)
    else:
        X1 = np.tensordot(Q3, T, axes=([0], [0]))  # [u,m,k,b]
        X2 = absorb_split(X1, A)                   # [m,b,d,j]
        T_raw = np.tensordot(X2, Q3, axes=([1, 2], [0, 1]))  # [m,j,n]
    Y = np.tensordot(T_raw, R, axes=([0], [0]))    # [j,n,g]
    C_raw = np.tensordot(Y, Q3, axes=([2, 0], [0, 1]))  # [n,p]
    C_new, T_new = sym_norm(C_raw, T_raw)
    return dict(ct=ct, Q=Q, R=R, T_raw=T_raw, C_raw=C_raw, C=C_new, T=T_new)


def qr_step(C, T, A, layers="double"):
    p = qr_step_parts(C, T, A, layers)
    return p["C"], p["T"]


# ---------------------------------------------------------------------------
# Convergence on the corner spectrum (Standard CTMRG paragraph: "repeated
# until convergence"; reading: change of the normalised |eig(C)|)
# ---------------------------------------------------------------------------

def corner_spectrum(C):
    """Sorted |eigenvalues| of the symmetric corner, descending."""
    Cr = np.real(C)
    w = np.linalg.eigvalsh(0.5 * (Cr + Cr.T))
    return np.sort(np.abs(w))[::-1]


def spectrum_delta(s_new, s_old):
    n = max(len(s_new), len(s_old))
    a = np.zeros(n)
    b = np.zeros(n)
    a[:len(s_new)] = s_new
    b[:len(s_old)] = s_old
    return float(np.sqrt(np.sum((a - b) ** 2)))


def warmup(A, chi, n_warmup=None, env=None, layers="double"):
    """Warm-up with standard steps, growing chi towards the target (QR-CTMRG
    paragraph: 1-4 standard steps suffice and let chi grow).  Reading: at
    least two steps, more if chi0 * D^(2n) < chi.  With ``layers='network'``
    A is the network tensor a itself (bond D2 = A.shape[0])."""
    if layers == "network":
        a = A
        C, T = init_env_network(a) if env is None else env
    else:
        a = double_layer(A)
        C, T = init_env(A) if env is None else env
    D2 = a.shape[0]
    if n_warmup is None:
        n_warmup, c = 0, C.shape[0]
        while c < chi:
            c *= D2
            n_warmup += 1
            if D2 == 1:
                break
        n_warmup = max(2, n_warmup)
    for _ in range(n_warmup):
        C, T = eigen_step(C, T, a, chi)
    return C, T


def ctmrg(A, chi, method="qr", tol=1e-12, max_iter=200, n_warmup=None,
          env=None, layers="double", check_every=1, init=None):
    """Run C4v CTMRG to convergence of the corner spectrum.

    ``method='qr'``: warm-up standard steps, then QR-CTMRG steps.
    ``method='eigen'``: standard steps throughout.  ``init`` (C, T) skips the
    warm-up.  ``layers='network'``: A is a classical network tensor a[u,l,d,r]
    used as it is (Discussion: classical partition functions).  Returns
    (C, T, info) with info['iters'], info['delta'], info['converged'] and the
    spectrum history.
    """
    a = A if layers == "network" else double_layer(A)
    if init is not None:
        C, T = init
    else:
        C, T = warmup(A, chi, n_warmup, env, layers)
    s_old = corner_spectrum(C)
    hist = []
    delta = np.inf
    it = 0
    for it in range(1, max_iter + 1):
        if method == "qr":
            C, T = qr_step(C, T, A, layers)
        else:
            C, T = eigen_step(C, T, a, chi)
        if it % check_every == 0:
            s = corner_spectrum(C)
            delta = spectrum_delta(s, s_old)
            hist.append(delta)
            s_old = s
            if delta < tol:
                break
    return C, T, dict(iters=it, delta=delta, converged=delta < tol, hist=hist)


# ---------------------------------------------------------------------------
# Observables (Results paragraphs: Heisenberg with a sublattice rotation,
# J1-J2 model)
# ---------------------------------------------------------------------------

def spin_ops():
    sx = np.array([[0, 1], [1, 0]], dtype=complex) / 2
    sy = np.array([[0, -1j], [1j, 0]], dtype=complex) / 2
    sz = np.array([[1, 0], [0, -1]], dtype=complex) / 2
    return sx, sy, sz


def heisenberg_bond():
    """h = S_1 . S_2 as a real 4x4 matrix on (s1 s2),(t1 t2)."""
    sx, sy, sz = spin_ops()
    h = np.kron(sx, sx) + np.kron(sy, sy) + np.kron(sz, sz)
    assert np.allclose(h.imag, 0)
    return h.real


def rotated_heisenberg_bond():
    """h~ = (1 x U)^dag h (1 x U), U = exp(i pi sigma^y / 2) on the second site
    (the sublattice rotation that makes the Neel state C4v ferromagnetic)."""
    sy = np.array([[0, -1j], [1j, 0]])
    U = np.cos(np.pi / 2) * np.eye(2) + 1j * np.sin(np.pi / 2) * sy
    W = np.kron(np.eye(2), U)
    hr = W.conj().T @ heisenberg_bond() @ W
    assert np.allclose(hr.imag, 0)
    return hr.real


def rdm_nn(C, T, A):
    """Two horizontally adjacent sites in a 2x1 patch (4 C, 6 T).

    rho[s1,t1,s2,t2]; the left half is
    HL[x,h,z,s,t] = sum L[x1,q,z1] T[x1,p,x] T[z1,P,z] aO[s,t,p,q,P,h]
    with L[x1,q,z1] = sum C[y1,x1] T[y1,q,y2] C[y2,z1]; the right half is
    its mirror image, joined on (x, h, z).
    """
    aO = double_layer_open(A)
    L = np.tensordot(np.tensordot(C, T, axes=([0], [0])), C, axes=([2], [0]))  # [x1,q,z1]
    W = np.tensordot(L, T, axes=([0], [0]))                  # [q,z1,p,X]
    W = np.tensordot(W, T, axes=([1], [0]))                  # [q,p,X,P,Z]
    HL = np.tensordot(W, aO, axes=([1, 0, 3], [2, 3, 4]))    # [X,Z,s,t,h]
    HL = np.transpose(HL, (0, 4, 1, 2, 3))                   # [X,h,Z,s,t]
    # right half: the mirror image, site legs (u=p, l=h, d=P, r=q)
    HR = np.tensordot(W, aO, axes=([1, 0, 3], [2, 5, 4]))    # [X,Z,s,t,h]
    HR = np.transpose(HR, (0, 4, 1, 2, 3))
    return np.tensordot(HL, HR, axes=([0, 1, 2], [0, 1, 2]))  # [s1,t1,s2,t2]


def enlarged_corner_open(C, T, A):
    """Ct_open[(b,l),(r,j),s,t]: enlarged corner with the site's physical legs open."""
    chi, D2 = T.shape[0], T.shape[1]
    d = A.shape[0]
    aO = double_layer_open(A)
    ct = np.tensordot(C, T, axes=([1], [0]))                 # [g,i,r]
    X = np.tensordot(ct, T, axes=([0], [0]))                 # [i,r,k,b]
    Ct = np.tensordot(X, aO, axes=([0, 2], [2, 3]))          # [r,b,s,t,l,j]
    Ct = np.transpose(Ct, (1, 4, 0, 5, 2, 3))                # [b,l,r,j,s,t]
    return Ct.reshape(chi * D2, chi * D2, d, d)


def rdm_nnn(C, T, A):
    """Two diagonal sites of a 2x2 patch (4 C, 8 T); the other two sites are
    traced.  rho[s1,t1,s4,t4] = Tr(Ct_open(s1,t1) Ct Ct_open(s4,t4) Ct): by
    C4v symmetry the four quadrants are the same enlarged corner."""
    a = double_layer(A)
    Ct = enlarged_corner(C, T, a)
    Co = enlarged_corner_open(C, T, A)
    P = np.tensordot(Co, Ct, axes=([1], [0]))                # [a,s,t,c]
    return np.tensordot(P, P, axes=([0, 3], [3, 0]))          # [s1,t1,s4,t4]


def bond_energy(rho4, h):
    """<h> = Tr(rho h) / Tr(rho) with rho[s1,t1,s2,t2] -> [(s1 s2),(t1 t2)]."""
    d = rho4.shape[0]
    rho = np.transpose(rho4, (0, 2, 1, 3)).reshape(d * d, d * d)
    return np.trace(rho @ h.T) / np.trace(rho)


def energy(C, T, A, J1=1.0, J2=0.0, rotate=True):
    """Energy per site: 2 J1 <h~>_nn + 2 J2 <h>_nnn (two NN and two NNN bonds
    per site; NN pairs use the sublattice-rotated bond, NNN pairs share a
    sublattice and use the plain bond).  rotate=False takes the plain bond on
    NN pairs too (no sublattice rotation)."""
    hnn = rotated_heisenberg_bond() if rotate else heisenberg_bond()
    E = 2.0 * J1 * bond_energy(rdm_nn(C, T, A), hnn)
    if J2 != 0.0:
        E = E + 2.0 * J2 * bond_energy(rdm_nnn(C, T, A), heisenberg_bond())
    return E


# ---------------------------------------------------------------------------
# Derivatives (Automatic differentiation paragraph; fixed-point AD named in
# the Discussion).  Complex step: d/de E(A + e v) = Im E(A + i h v) / h.
# ---------------------------------------------------------------------------

def env_change(C1, T1, C2, T2):
    return float(np.sqrt(np.sum(np.abs(C1 - C2) ** 2) + np.sum(np.abs(T1 - T2) ** 2)))


def complex_spectrum(C):
    """Eigenvalues of a (complex) symmetric corner ordered by |Re|, descending.
    For C = C_r + i h C_i the imaginary parts carry the first-order change of
    the spectrum, so convergence of both parts is gauge invariant."""
    w = np.linalg.eigvals(C)
    return w[np.argsort(-np.abs(np.real(w)), kind="stable")]


def fixed_point_env(A, C, T, tol=1e-13, max_iter=2000, h=None, layers="double"):
    """Iterate QR steps from (C, T) until the corner spectrum stops changing.

    The QR map is covariant under orthogonal gauge changes of the chi legs and
    alternates a sign gauge between steps, so the test is on the spectrum, not
    on the entries.  With complex input (a complex step of size ``h``) the
    imaginary parts are tested relative to ``h``.  An even number of steps is
    always taken.
    """
    s_old = complex_spectrum(C)
    ch = np.inf
    it = 0
    for it in range(2, max_iter + 1, 2):
        C, T = qr_step(C, T, A, layers)
        C, T = qr_step(C, T, A, layers)
        s = complex_spectrum(C)
        n = min(len(s), len(s_old))
        ch = float(np.max(np.abs(np.real(s[:n] - s_old[:n]))))
        if h is not None:
            ch = max(ch, float(np.max(np.abs(np.imag(s[:n] - s_old[:n])))) / h)
        s_old = s
        if ch < tol:
            break
    return C, T, dict(iters=it, change=ch)


def directional_derivative_fixed_point(A, v, C, T, J1=1.0, J2=0.0,
                                       h=1e-20, tol=1e-13, max_iter=2000):
    """dE/dA . v at the converged environment, by complex step through the
    QR-CTMRG fixed point started from the real converged (C, T)."""
    Ac = A.astype(complex) + 1j * h * v
    Cc, Tc, info = fixed_point_env(Ac, C.astype(complex), T.astype(complex),
                                   tol=tol, max_iter=max_iter, h=h)
    return float(np.imag(energy(Cc, Tc, Ac, J1, J2)) / h), info


def directional_derivative_unrolled(A, v, C, T, k, J1=1.0, J2=0.0, h=1e-20, layers="double",
                                    rotate=True):
    """dE/dA . v of E(A, F^k(A; C, T)) with (C, T) held fixed: the gradient of
    k tracked CTMRG steps started from a detached environment.  ``layers``
    picks the double-layer or the ket-then-bra form of the edge update (equal
    up to rounding; the second is cheaper for D >= 3)."""
    Ac = A.astype(complex) + 1j * h * v
    Cc, Tc = C.astype(complex), T.astype(complex)
    for _ in range(k):
        Cc, Tc = qr_step(Cc, Tc, Ac, layers)
    return float(np.imag(energy(Cc, Tc, Ac, J1, J2, rotate)) / h)


def energy_at(A, C, T, J1=1.0, J2=0.0, tol=1e-13, max_iter=2000):
    """E(A) with the environment re-converged from (C, T) (used for FD)."""
    Cc, Tc, _ = fixed_point_env(A, C, T, tol=tol, max_iter=max_iter)
    return float(np.real(energy(Cc, Tc, A, J1, J2)))


# ---------------------------------------------------------------------------
# Classical 2D Ising model as a C4v network (Discussion: QR-CTMRG applies to
# classical partition functions)
# ---------------------------------------------------------------------------

def ising_A(beta):
    """A[s,u,l,d,r] = W[s,u] W[s,l] W[s,d] W[s,r], W = B^(1/2),
    B = exp((beta/2) s s').  Then sum_{r,r'} of the ket/bra bond weights
    between neighbours is B[s1,s2]^2 = exp(beta s1 s2): the double layer a is
    the Ising network at inverse temperature beta (index 0 is s=+1)."""
    spins = np.array([1.0, -1.0])
    B = np.exp(0.5 * beta * np.outer(spins, spins))
    w, V = np.linalg.eigh(B)
    W = (V * np.sqrt(w)) @ V.T
    return np.einsum("su,sl,sd,sr->suldr", W, W, W, W)


def ising_kappa(C, T, a, a_obs=None):
    """Partition function per site kappa = Z11 Z00 / Z10^2 (normalisations of
    C and T cancel).  With ``a_obs`` returns <O> = Z11(a_obs) / Z11(a).
    Nothing here is specific to the Ising model: any C4v network tensor a
    (bond = C4v edge leg of T) works; ``network_kappa`` is the same function.

    Z00 = Tr C^4 (four corners), Z10 = a 2x1 ring C T C C T C, Z11 = the
    3x3 patch (four C, four T, one a)."""
    Z00 = np.trace(C @ C @ C @ C)
    Z10 = np.einsum("yx,xkX,XY,YZ,ZkW,Wy->", C, T, C, C, T, C, optimize="greedy")

    def z11(t):
        return np.einsum("ax,xpy,yb,bqc,cz,zrw,wd,dsa,psrq->",
                         C, T, C, T, C, T, C, T, t, optimize="greedy")
    Z11 = z11(a)
    if a_obs is not None:
        return z11(a_obs) / Z11
    return Z11 * Z00 / Z10 ** 2


network_kappa = ising_kappa


def spin_network(B, obs=None):
    """Classical network tensor of spins with Boltzmann weight B[s,s'] on
    every bond (B symmetric positive definite):
        a[u,l,d,r] = sum_s o[s] W[s,u] W[s,l] W[s,d] W[s,r],  W = B^(1/2),
    o = 1 (the network) or ``obs`` (the same network with o[s] inserted at
    one site).  Neighbouring tensors share one bond index r, and
    sum_r W[s1,r] W[s2,r] = B[s1,s2], so the contracted network is the
    partition function; a is C4v symmetric and its bond is q = len(B).
    B may be semidefinite (beta = 0): eigenvalues below 0 by rounding are
    taken as 0."""
    w, V = np.linalg.eigh(B)
    W = (V * np.sqrt(np.maximum(w, 0.0))) @ V.T
    o = np.ones(B.shape[0]) if obs is None else np.asarray(obs, dtype=float)
    return np.einsum("s,su,sl,sd,sr->uldr", o, W, W, W, W), W


def ising_network(beta):
    """Ising network with bond 2: B = exp(beta s s'), s = +1, -1 (index 0 is
    +1).  Returns (a, a_sigma, W)."""
    spins = np.array([1.0, -1.0])
    B = np.exp(beta * np.outer(spins, spins))
    a, W = spin_network(B)
    a_s, _ = spin_network(B, spins)
    return a, a_s, W


def potts_network(q, beta):
    """q-state Potts network with bond q: B = exp(beta delta_{s s'}).
    Returns (a, W)."""
    B = np.exp(beta * np.eye(q))
    return spin_network(B)


def init_env_network(a, v=None):
    """Boundary tensors of a network fed directly: the legs that point out of
    the system are contracted with the vector v (all ones when None, i.e. a
    free boundary):
        C0[d,r]   = sum_{u,l} v[u] v[l] a[u,l,d,r],
        T0[u,r,d] = sum_l v[l] a[u,l,d,r]
    (the same leg assignment as ``init_env``), then sym_norm."""
    b = a.shape[0]
    v = np.ones(b) if v is None else np.asarray(v, dtype=float)
    C0 = np.einsum("u,l,uldr->dr", v, v, a)
    T0 = np.einsum("l,uldr->urd", v, a)
    return sym_norm(C0, T0)


def ising_observable_layer(A):
    """a_sigma = sum_s s A[s] (x) A[s]: the double layer with the spin inserted."""
    D = A.shape[1]
    spins = np.array([1.0, -1.0])
    a = np.einsum("s,suldr,sULDR->uUlLdDrR", spins, A, A)
    return a.reshape(D * D, D * D, D * D, D * D)


def onsager_free_energy(beta, n=512):
    """-beta f = ln 2 + 1/(8 pi^2) int_0^{2pi} int_0^{2pi}
    ln[cosh^2(2b) - sinh(2b)(cos t1 + cos t2)] (midpoint rule on the periodic
    square: spectrally accurate away from the critical point, and it never
    samples the integrable log singularity at t1 = t2 = 0 of the critical
    point)."""
    t = 2 * np.pi * (np.arange(n) + 0.5) / n
    c = np.cos(t)
    arg = np.cosh(2 * beta) ** 2 - np.sinh(2 * beta) * (c[:, None] + c[None, :])
    return np.log(2.0) + 0.5 * np.mean(np.log(arg))


def yang_magnetization(beta):
    """Spontaneous magnetisation (1 - sinh(2 beta)^-4)^(1/8) below T_c."""
    s = np.sinh(2 * beta)
    return (1.0 - s ** -4) ** 0.125 if s > 1 else 0.0


# ---------------------------------------------------------------------------
# Variational optimisation (Automatic differentiation paragraph): L-BFGS on
# E(A); each evaluation runs two CTMRG steps without gradient tracking, then
# k tracked steps, the energy and its gradient; the boundary tensors of the
# previous step are reused except during the line search.
# ---------------------------------------------------------------------------

def c4v_orbit_basis(d, D):
    """Orthonormal basis of the C4v-invariant tensors A[s,u,l,d,r]: one
    indicator per orbit of index tuples under the eight leg permutations,
    divided by the square root of the orbit size.  Its length is n(D) of the
    iPEPS footnote."""
    seen = np.zeros((d, D, D, D, D), dtype=bool)
    basis = []
    for idx in np.ndindex(d, D, D, D, D):
        if seen[idx]:
            continue
        s, legs = idx[0], idx[1:]
        orbit = {(s,) + tuple(legs[p[i]] for i in range(4)) for p in C4V_PERMS}
        v = np.zeros((d, D, D, D, D))
        for o_idx in orbit:
            v[o_idx] = 1.0
            seen[o_idx] = True
        basis.append(v / np.sqrt(len(orbit)))
    return basis


def unrolled_energy_grad(A, C, T, k, J1=1.0, J2=0.0, h=1e-20, layers="double"):
    """E(A, F^k(A; C, T)) with (C, T) detached, its C4v gradient (one complex
    step along every orbit basis vector: g = sum_O (dE . v_O) v_O = sym(dE)),
    and the environment after the k steps."""
    Ck, Tk = C, T
    for _ in range(k):
        Ck, Tk = qr_step(Ck, Tk, A, layers)
    E = float(np.real(energy(Ck, Tk, A, J1, J2)))
    g = np.zeros_like(A)
    for v in c4v_orbit_basis(A.shape[0], A.shape[1]):
        Ac = A.astype(complex) + 1j * h * v
        Cc, Tc = C.astype(complex), T.astype(complex)
        for _ in range(k):
            Cc, Tc = qr_step(Cc, Tc, Ac, layers)
        g = g + (float(np.imag(energy(Cc, Tc, Ac, J1, J2))) / h) * v
    return E, g, Ck, Tk


def lbfgs_direction(g, pairs):
    """p = -H g by the L-BFGS two-loop recursion over the stored pairs
    (s, y), oldest first, with H0 = (s.y / y.y) I from the newest pair
    (Nocedal and Wright, Numerical Optimization, two-loop recursion)."""
    q = g.copy()
    alphas = []
    for s, y in reversed(pairs):
        a = np.sum(s * q) / np.sum(y * s)
        alphas.append(a)
        q = q - a * y
    if pairs:
        s, y = pairs[-1]
        q = q * (np.sum(s * y) / np.sum(y * y))
    for (s, y), a in zip(pairs, reversed(alphas)):
        b = np.sum(y * q) / np.sum(y * s)
        q = q + (a - b) * s
    return -q


def lbfgs_minimize(evaluate, x0, n_steps, history=10, step0=0.1, c1=1e-4, max_ls=10,
                   accept=None):
    """L-BFGS with a backtracking Armijo line search.

    ``evaluate(x, trial) -> (f, g)``; ``trial`` is 0 for the starting point
    and for the first point tried in a step, >= 1 for the later points of a
    line search.  Readings (the paper names L-BFGS only): the first step has
    length ``step0`` along -g, later steps start at alpha = 1; a point is
    accepted when f <= f_k + c1 alpha g.p, else alpha is halved, at most
    ``max_ls`` points per step; a pair (s, y) is kept when s.y > 1e-10 |s||y|;
    a direction that is not a descent direction resets the history.
    ``accept()`` is called after a point is accepted; the loop ends early at
    a zero gradient.  Returns (x, energies, evaluations, line_search_failed).
    """
    x = x0.copy()
    f, g = evaluate(x, 0)
    if accept:
        accept()
    fs, nev, pairs = [f], 1, []
    for _ in range(n_steps):
        if not np.any(g):
            break                        # stationary point: no direction
        p = lbfgs_direction(g, pairs)
        gp = float(np.sum(g * p))
        if not gp < 0:
            pairs = []
            p = -g
            gp = float(np.sum(g * p))
        alpha = 1.0 if pairs else step0 / float(np.sqrt(np.sum(p * p)))
        ok = False
        for t in range(max_ls):
            xt = x + alpha * p
            ft, gt = evaluate(xt, t)
            nev += 1
            if ft <= f + c1 * alpha * gp:
                ok = True
                break
            alpha *= 0.5
        if not ok:
            return x, fs, nev, True
        if accept:
            accept()
        s, y = xt - x, gt - g
        if np.sum(s * y) > 1e-10 * np.sqrt(np.sum(s * s) * np.sum(y * y)):
            pairs = (pairs + [(s, y)])[-history:]
        x, f, g = xt, ft, gt
        fs.append(f)
    return x, fs, nev, False


def optimize_ipeps(A0, chi, J1=1.0, J2=0.0, n_steps=5, k=10, nograd=2, history=10,
                   step0=0.1, c1=1e-4, max_ls=10, env_tol=1e-12, env_max_iter=2000):
    """L-BFGS on the energy per site (Automatic differentiation paragraph).

    An evaluation at A takes the environment of the last accepted point
    (trial 0 of a step) or a fresh one, converged from the bulk boundary
    (start, and the later points of a line search); runs ``nograd`` QR-CTMRG
    steps, then the energy and gradient of ``k`` tracked steps.  The
    environment after the tracked steps is what the next step reuses."""
    layers = "double"
    state = {"env": None, "cand": None}

    def evaluate(A, trial):
        if trial == 0 and state["env"] is not None:
            C, T = state["env"]
        else:
            C, T, _ = ctmrg(A, chi, "qr", tol=env_tol, max_iter=env_max_iter, check_every=5)
        for _ in range(nograd):
            C, T = qr_step(C, T, A, layers)
        E, g, Ck, Tk = unrolled_energy_grad(A, C, T, k, J1, J2, layers=layers)
        state["cand"] = (Ck, Tk)
        return E, g

    def accept():
        state["env"] = state["cand"]

    return lbfgs_minimize(evaluate, A0, n_steps, history, step0, c1, max_ls, accept)
