"""Plain, slow FP64 / complex128 CPU oracle for block belief propagation (blockBP).

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py``.  The product path (the CUDA library behind ``include/bbp.h``) never
imports, links or executes anything here, and this module imports nothing from
the product package.

Every function names the passage of Guo, Poletti & Arad, "Block belief propagation
algorithm for two-dimensional tensor networks" (arXiv:2301.05844) that it follows.
Where the paper is silent the reading taken is stated in the docstring.

Conventions
-----------
* PEPS site tensor ``T[p, u, l, d, r]`` (physical, up, left, down, right).  With open
  boundaries (OBC) the legs on the lattice edge have dimension 1 (Sec. "The blockBP
  algorithm": an OBC PEPS is a PBC PEPS with bond dimension 1 at the boundary).
* Double-layer tensor ``E[u, l, d, r]`` with every leg the merged (ket, bra) pair,
  merged index ``ket * D + bra`` (Fig. 1(a,b)).
* MPS site ``M[a, k, b]`` (left bond, physical, right bond).  MPO site
  ``O[w, p, q, w']`` (left MPO bond, input physical, output physical, right MPO bond).
* A block message is an open MPS along the shared block edge, sites ordered top to
  bottom on vertical edges and left to right on horizontal edges.
* Directions: LEFT=0, RIGHT=1, UP=2, DOWN=3.

Nothing here is blocked, fused or reordered beyond the definitions; numpy's
``einsum`` / ``linalg.qr`` serve as library primitives.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LEFT, RIGHT, UP, DOWN = 0, 1, 2, 3
OPPOSITE = {LEFT: RIGHT, RIGHT: LEFT, UP: DOWN, DOWN: UP}

# --------------------------------------------------------------------------------------
# Counter-based generator.  The paper draws the initial fit MPS at random (App. A,
# "initializing |Y> randomly").  Both this oracle and the CUDA library implement the
# same published generator, SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), keyed by
# (seed, stream, index), so the two sides start every fit from identical numbers.
#   key   = splitmix64(seed XOR splitmix64(stream))
#   z_i   = splitmix64(key + i)                      (all arithmetic mod 2^64)
#   u_i   = (z_i >> 11) * 2^-52 - 1                  (exact double in [-1, 1))
# --------------------------------------------------------------------------------------
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MUL1 = np.uint64(0xBF58476D1CE4E5B9)
_MUL2 = np.uint64(0x94D049BB133111EB)


def splitmix64(z):
    """One SplitMix64 output step applied elementwise to uint64 values. (The published SplitMix64 step of Steele, Lea & Flood: the paper draws the fits' initial states at random without naming a generator, App. A, so both implementations use this counter-based one.)"""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _MUL1
        z = (z ^ (z >> np.uint64(27))) * _MUL2
    return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, stream: int, n: int) -> np.ndarray:
    """n exact doubles in [-1, 1) from the counter-based generator. (App. A draws the fits' initial states at random; these uniforms are that draw.)"""
    key = splitmix64(np.uint64(seed) ^ splitmix64(np.uint64(stream)))
    with np.errstate(over="ignore"):
        z = splitmix64(key + np.arange(n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0


def stream_id(tag: int, outer: int, msg: int, col: int, site: int) -> int:
    """Pack the identity of one fit-initial site into a 64-bit stream number.

    tag 0 = message update (outer = BP sweep index, msg = 4*block + direction);
    tag 1 = read-out environment (outer = region id, msg = 0 right env, 1 left env).
    (One stream per fit-initial site, so that every implementation draws the same numbers.)
    """
    assert site < 256 and col < 256 and msg < (1 << 20) and outer < (1 << 20) and tag < 256
    return (tag << 56) | (outer << 36) | (msg << 16) | (col << 8) | site


def random_site(seed: int, stream: int, shape, dtype) -> np.ndarray:
    """Fit-initial site tensor: C-order fill; complex entries interleave (re, im). (App. A: each fit starts from a random MPS.)"""
    n = int(np.prod(shape))
    if np.issubdtype(dtype, np.complexfloating):
        v = uniform_pm1(seed, stream, 2 * n)
        return (v[0::2] + 1j * v[1::2]).reshape(shape)
    return uniform_pm1(seed, stream, n).reshape(shape)


# --------------------------------------------------------------------------------------
# Double layer (Sec. "The blockBP algorithm", Fig. 1(a,b)).
# --------------------------------------------------------------------------------------
def double_layer(T: np.ndarray, O: np.ndarray | None = None) -> np.ndarray:
    """E[(u u'),(l l'),(d d'),(r r')] = sum_{p,p'} O[p',p] T[p,u,l,d,r] conj(T[p',u',l',d',r']).

    Contracting the physical legs of ket and bra gives the closed network for
    <psi|psi>; with a local operator O between them it gives <psi|O|psi>.
    O=None means the identity.  Merged leg index = ket * D + bra.
    (Fig. 1(a,b).)
    """
    d, Du, Dl, Dd, Dr = T.shape
    OT = T if O is None else np.einsum("qp,puldr->quldr", O, T)
    E = np.einsum("quldr,qULDR->uUlLdDrR", OT, np.conj(T))
    return E.reshape(Du * Du, Dl * Dl, Dd * Dd, Dr * Dr)


def hermitian_basis_matrix(D: int) -> np.ndarray:
    """Unitary V on a merged (ket a, bra b) leg, k = a * D + b, whose rows give the coordinates
    v_(a,a) at k = a*D+a, (v_(a,b) + v_(b,a)) / sqrt 2 at k = a*D+b for a < b, and
    (v_(b,a) - v_(a,b)) / (i sqrt 2) at k = a*D+b for a > b.

    Not a step of the paper: a fixed change of basis on every leg of the double layer
    (Fig. 1(b)) in which a vector that is Hermitian under the swap of ket and bra has real
    coordinates.  Up and left legs take V, down and right legs conj(V), so that every bond
    contracts through V^T conj(V) = I and each contraction keeps its value."""
    V = np.zeros((D * D, D * D), dtype=np.complex128)
    h = 1.0 / math.sqrt(2.0)
    for a in range(D):
        for b in range(D):
            k, kt = a * D + b, b * D + a
            if a == b:
                V[k, k] = 1.0
            elif a < b:
                V[k, k] = h
                V[k, kt] = h
            else:
                V[k, kt] = h / 1j
                V[k, k] = -h / 1j
    return V


def to_hermitian_basis_E(E: np.ndarray, Dims) -> np.ndarray:
    """E[u, l, d, r] with V on the up and left legs and conj(V) on the down and right legs
    (the double layer in the Hermitian basis; real when E is Hermitian under the joint swap
    of ket and bra on all legs)."""
    Du, Dl, Dd, Dr = Dims
    Vs = [hermitian_basis_matrix(Du), hermitian_basis_matrix(Dl),
          np.conj(hermitian_basis_matrix(Dd)), np.conj(hermitian_basis_matrix(Dr))]
    out = np.asarray(E, dtype=np.complex128)
    for leg, V in enumerate(Vs):  # one leg at a time: out[..., K, ...] = sum_k V[K, k] out[..., k, ...]
        out = np.moveaxis(np.tensordot(V, out, axes=([1], [leg])), 0, leg)
    return out


def to_hermitian_basis_mps(M, D: int, conj_basis: bool):
    """Message sites [a, k, b] with V (conj(V) when conj_basis) on every physical leg."""
    V = hermitian_basis_matrix(D)
    if conj_basis:
        V = np.conj(V)
    return [np.einsum("Kk,akb->aKb", V, s) for s in M]


# --------------------------------------------------------------------------------------
# Orthonormal factors with diag(R) real and >= 0 (App. A, QR on the left-to-right
# half sweep, LQ on the right-to-left half sweep; only the orthonormal factor is kept).
# --------------------------------------------------------------------------------------
def qr_q(M: np.ndarray) -> np.ndarray:
    """Thin Q of M (m x n, m >= n) with the diagonal of R made real non-negative. (App. A: the left-to-right half sweep keeps Q of a QR.)"""
    Q, R = np.linalg.qr(M, mode="reduced")
    dg = np.diag(R)
    ph = np.ones_like(dg)
    nz = np.abs(dg) > 0
    ph[nz] = dg[nz] / np.abs(dg[nz])
    return Q * ph[None, :]


def lq_q(M: np.ndarray) -> np.ndarray:
    """Row-orthonormal Q of M = L Q (m x n, m <= n), diag(L) real non-negative. (App. A: the right-to-left half sweep keeps Q of an LQ.)"""
    return qr_q(np.conj(M.T)).conj().T


# --------------------------------------------------------------------------------------
# Variational MPO x MPS fit (App. A, Eq. "distance" and Eq. "update", Fig. S1).
# --------------------------------------------------------------------------------------
def site_update(A, O, X, B):
    """Eq. (update): Yt[y,q,y'] = sum A[y,w,x] X[x,p,x'] O[w,p,q,w'] B[y',w',x'].

    Evaluated as three pairwise tensordot contractions (x, then w and p, then x' and w')."""
    t = np.tensordot(A, X, axes=([2], [0]))              # [y, w, p, x']
    t = np.tensordot(t, O, axes=([1, 2], [0, 1]))        # [y, x', q, w']
    return np.tensordot(t, B, axes=([1, 3], [2, 1]))     # [y, q, y']


def env_left(A, Y, O, X):
    """Left-environment recurrence of App. A: A_{l+1}[y',w',x'] =
    sum A_l[y,w,x] conj(Y[y,q,y']) O[w,p,q,w'] X[x,p,x']."""
    t = np.tensordot(A, X, axes=([2], [0]))              # [y, w, p, x']
    t = np.tensordot(t, O, axes=([1, 2], [0, 1]))        # [y, x', q, w']
    t = np.tensordot(np.conj(Y), t, axes=([0, 1], [0, 2]))  # [y', x', w']
    return t.transpose(0, 2, 1)


def env_right(B, Y, O, X):
    """Right-environment recurrence of App. A: B_l[y,w,x] =
    sum conj(Y[y,q,y']) O[w,p,q,w'] X[x,p,x'] B_{l+1}[y',w',x']."""
    t = np.tensordot(X, B, axes=([2], [2]))              # [x, p, y', w']
    t = np.tensordot(t, O, axes=([1, 3], [1, 3]))        # [x, y', w, q]
    t = np.tensordot(np.conj(Y), t, axes=([1, 2], [3, 1]))  # [y, x, w]
    return t.transpose(0, 2, 1)


def bond_caps(phys, chi):
    """Bond dimensions of an n-site MPS with physical dims phys, capped at chi:
    bond_i = min(chi, prod(phys[:i]), prod(phys[i:])), ends 1. (App. A: the bonds of a boundary MPS are capped at chi.)"""
    n = len(phys)
    b = [1]
    for i in range(1, n):
        b.append(min(chi, math.prod(phys[:i]), math.prod(phys[i:])))
    b.append(1)
    return b


@dataclass
class FitOpts:
    """Zip-up fit controls (App. A): tolerance on std/|mean| of the per-update losses
    over one full sweep, and the maximum number of sweeps."""
    chi: int
    tol: float = 1e-6
    max_sweeps: int = 10


def fit_mpo_mps(O, X, opts: FitOpts, init_site, dtype):
    """Variational fit of a bond-chi MPS Y to O|X> (App. A).

    Y starts at random with bonds at their caps; the right environments are built
    from that Y directly (App. A builds B from the initial Y, with A_1 = B_{L+1} = 1).
    One sweep = left-to-right over sites 0..n-2 (update, QR, keep Q, update A) then
    right-to-left over n-1..1 (update, LQ, keep Q, update B).  The loss of each update
    is -||Yt||^2; the sweep loop stops when std/|mean| over one sweep < tol, or after
    max_sweeps.  A last update at site 0 keeps Yt itself, so Y carries the norm.
    Returns (Y, list of per-sweep loss lists).
    """
    n = len(X)
    qd = [o.shape[2] for o in O]
    bonds = bond_caps(qd, opts.chi)
    Y = [init_site(i, (bonds[i], qd[i], bonds[i + 1])).astype(dtype) for i in range(n)]
    one = np.ones((1, 1, 1), dtype=dtype)
    A = [None] * (n + 1)
    B = [None] * (n + 1)
    A[0] = one
    B[n] = one
    for i in range(n - 1, 0, -1):
        B[i] = env_right(B[i + 1], Y[i], O[i], X[i])
    history = []
    for _ in range(opts.max_sweeps):
        losses = []
        for i in range(0, n - 1):
            Yt = site_update(A[i], O[i], X[i], B[i + 1])
            losses.append(-float(np.vdot(Yt, Yt).real))
            a, q, b = Yt.shape
            Y[i] = qr_q(Yt.reshape(a * q, b)).reshape(a, q, b)
            A[i + 1] = env_left(A[i], Y[i], O[i], X[i])
        for i in range(n - 1, 0, -1):
            Yt = site_update(A[i], O[i], X[i], B[i + 1])
            losses.append(-float(np.vdot(Yt, Yt).real))
            a, q, b = Yt.shape
            Y[i] = lq_q(Yt.reshape(a, q * b)).reshape(a, q, b)
            B[i] = env_right(B[i + 1], Y[i], O[i], X[i])
        history.append(losses)
        mean = float(np.mean(losses))
        if mean != 0.0 and float(np.std(losses)) / abs(mean) < opts.tol:
            break
    Y[0] = site_update(A[0], O[0], X[0], B[1])
    return Y, history


# --------------------------------------------------------------------------------------
# MPS utilities.
# --------------------------------------------------------------------------------------
def mps_overlap(M1, M2):
    """<M1|M2> for two MPS with equal physical dims (conj on M1). (Used for norms and the residual, Sec. "The blockBP algorithm", stop rule.)"""
    t = np.ones((1, 1), dtype=np.result_type(M1[0], M2[0]))
    for a, b in zip(M1, M2):
        t = np.tensordot(t, np.conj(a), axes=([0], [0]))      # [b_, k, c]
        t = np.tensordot(t, b, axes=([0, 1], [0, 1]))         # [c, d]
    return t[0, 0]


def mps_reverse(M):
    """Mirror an MPS: site order reversed, each site's two bonds swapped. (Used to rotate a block so that every outgoing message is computed as a left message.)"""
    return [s.transpose(2, 1, 0) for s in reversed(M)]


def identity_trace(M, D):
    """<I|m>: contract every site's merged (ket, bra) leg with delta_{ket,bra}. (The phase reference of a message: the paper fixes no phase, and <I|m> is made real positive.)"""
    t = np.ones((1,), dtype=M[0].dtype)
    for s in M:
        a, k, b = s.shape
        Dk = int(round(math.sqrt(k)))
        diag = s.reshape(a, Dk, Dk, b)[:, np.arange(Dk), np.arange(Dk), :].sum(axis=1)
        t = t @ diag
    return t[0]


def ones_trace(M):
    """<1|m>: contract every site's physical leg with the all-ones vector (the phase
    reference of a single-layer network, whose legs carry no (ket, bra) pair)."""
    t = np.ones((1,), dtype=M[0].dtype)
    for s in M:
        t = t @ s.sum(axis=1)
    return t[0]


def normalise_message(M, D, single=False):
    """Unit 2-norm, then the phase/sign fixed so that <I|m> is real positive.

    The paper normalises messages before comparing them (Sec. "The blockBP
    algorithm", stop rule) without naming the norm; the 2-norm and the identity-trace
    phase are the readings taken.  The phase is left alone when |<I|m>| < 1e-14.
    single: the message of a single-layer network, whose phase reference is <1|m>
    (the all-ones vector on every site) instead.
    """
    M = [s.copy() for s in M]
    nrm = math.sqrt(max(float(mps_overlap(M, M).real), 0.0))
    if not np.isfinite(nrm) or nrm == 0.0:
        raise FloatingPointError("zero-norm or non-finite message")
    M[0] = M[0] / nrm
    tau = ones_trace(M) if single else identity_trace(M, D)
    if abs(tau) > 1e-14:
        M[0] = M[0] * (np.conj(tau) / abs(tau))
    return M


def embed_at_caps(M, chi):
    """The same MPS with every bond zero-padded to the capped dimension
    min(chi, K^i, K^(n-i)): message storage has the shape of a bond-chi message from
    the start (the state is unchanged)."""
    K = M[0].shape[1]
    caps = bond_caps([K] * len(M), chi)
    out = []
    for i, s in enumerate(M):
        a, k, b = s.shape
        t = np.zeros((caps[i], k, caps[i + 1]), dtype=s.dtype)
        t[:a, :, :b] = s
        out.append(t)
    return out


def trivial_mps(n, dtype):
    """Message from outside an OBC lattice: the scalar 1 on every (dimension-1) leg. (Sec. "The blockBP algorithm": an OBC lattice is a periodic one with bonds of dimension 1 on the boundary.)"""
    return [np.ones((1, 1, 1), dtype=dtype) for _ in range(n)]


def identity_message(n, D, dtype):
    """Product of delta_{ket,bra} on every site, bond 1 (init mode 0). (App. A starts the messages from a chosen state.)"""
    v = np.eye(D, dtype=dtype).reshape(1, D * D, 1)
    return [v.copy() for _ in range(n)]


def random_mpdo_message(n, D, seed, stream, dtype):
    """Init mode 1: product of random positive matrices G G^dagger (bond 1), G with
    normal entries (App. A initialises messages as a random MPDO with normal entries).
    Normal numbers come from the counter-based uniforms by the Box-Muller transform."""
    out = []
    for i in range(n):
        u = uniform_pm1(seed, stream + i, 2 * D * D)
        u1 = (u[0::2] + 1.0) * 0.5  # [0,1)
        u2 = (u[1::2] + 1.0) * 0.5
        g = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
        G = g.reshape(D, D).astype(dtype)
        out.append((G @ np.conj(G.T)).reshape(1, D * D, 1))
    return out


def ones_message(n, K, dtype):
    """Single-layer network, init mode 0: the all-ones vector on every site, bond 1. (The deterministic alternative to the uniform random start the paper uses for single-layer messages.)"""
    return [np.ones((1, K, 1), dtype=dtype) for _ in range(n)]


def uniform_message(n, K, seed, stream, dtype):
    """Single-layer network, init mode 1: a product message with independent uniform
    entries in [0, 1) on every site, bond 1 (the paper starts the message passing of a
    single-layer network from uniform random messages, Sec. on the 2D Ising model).  The
    uniforms are the counter-based ones, (u + 1) / 2 for u in [-1, 1)."""
    return [((uniform_pm1(seed, stream + i, K) + 1.0) * 0.5).astype(dtype).reshape(1, K, 1) for i in range(n)]


# --------------------------------------------------------------------------------------
# Frames: every outgoing direction is computed as the LEFT message of a rotated block.
# --------------------------------------------------------------------------------------
def frame(Eblk, m_in, direction):
    """Rotate a block so that `direction` becomes LEFT.

    Eblk: rows x cols list of double-layer tensors E[u,l,d,r].
    m_in: dict dir -> incoming message into the block from that side.
    Returns (E' grid, mT', mR', mB') in the rotated frame.  The left message of that
    frame, sites in frame row order, is the outgoing message in its natural order.
    Contraction then runs column by column from the frame's right edge to its left
    edge (App. A contracts right to left for the left message; the other three
    directions use the rotated equivalent).
    """
    H, W = len(Eblk), len(Eblk[0])
    if direction == LEFT:
        return [list(r) for r in Eblk], m_in[UP], m_in[RIGHT], m_in[DOWN]
    if direction == RIGHT:  # mirror left <-> right
        E2 = [[Eblk[r][W - 1 - c].transpose(0, 3, 2, 1) for c in range(W)] for r in range(H)]
        return E2, mps_reverse(m_in[UP]), m_in[LEFT], mps_reverse(m_in[DOWN])
    if direction == UP:  # transpose rows <-> cols
        E2 = [[Eblk[c][r].transpose(1, 0, 3, 2) for c in range(H)] for r in range(W)]
        return E2, m_in[LEFT], m_in[DOWN], m_in[RIGHT]
    if direction == DOWN:  # flip up <-> down, then transpose
        E2 = [[Eblk[H - 1 - c][r].transpose(1, 2, 3, 0) for c in range(H)] for r in range(W)]
        return E2, mps_reverse(m_in[LEFT]), m_in[UP], mps_reverse(m_in[RIGHT])
    raise ValueError(direction)


def column_mpo(Ef, mT, mB, c):
    """MPO for frame column c: [top message site, E[0,c], ..., E[H-1,c], bottom site].

    Horizontal legs run right (input) to left (output); vertical MPO bonds are the
    u/d legs.  Top site: O[1, alpha_{c+1}, alpha_c, v] = mT[c][alpha_c, v, alpha_{c+1}].
    Bottom site: O[v, beta_{c+1}, beta_c, 1] = mB[c][beta_c, v, beta_{c+1}].
    (App. A: one column of the block is applied as an MPO to the boundary MPS, Fig. 1(c).)
    """
    H = len(Ef)
    O = [mT[c].transpose(2, 0, 1)[None]]
    O += [Ef[r][c].transpose(0, 3, 1, 2) for r in range(H)]
    O += [mB[c].transpose(1, 2, 0)[..., None]]
    return O


def column_sweep(Ef, mT, mR, mB, opts: FitOpts, seed, stream_of, dtype, keep=False, warm=None, counts=None):
    """bMPS contraction of a block (frame) with its incoming messages (App. A, Fig. 1(d)).

    X starts as [1, mR, 1] (corner sites of dimension 1), then every column from the
    right edge to the left edge is absorbed by the zip-up fit with bond chi.  After
    each column the fitted MPS is scaled to unit norm (it is in mixed canonical form
    around site 0, so its norm is the Frobenius norm of site 0); the fits are
    scale-covariant, so this only removes over/underflow.
    warm (optional dict c -> site list): start column c's fit from that MPS instead of
    the random state (warm start from the previous sweep's fit of the same column);
    it is updated in place with every column's fitted MPS.
    counts (optional list): receives the number of fit sweeps each column's fit ran.
    Returns (list of column MPS after absorbing columns >= c, indexed by c) if keep,
    else the final column MPS.
    """
    H, W = len(Ef), len(Ef[0])
    one = np.ones((1, 1, 1), dtype=dtype)
    X = [one] + [s.astype(dtype) for s in mR] + [one]
    kept = {W: X}
    for c in range(W - 1, -1, -1):
        O = column_mpo(Ef, mT, mB, c)
        if warm is not None and c in warm:
            prev = warm[c]
            init = lambda i, shp, prev=prev, c=c: (prev[i].copy() if prev[i].shape == tuple(shp)
                                                   else random_site(seed, stream_of(c, i), shp, dtype))
        else:
            init = lambda i, shp: random_site(seed, stream_of(c, i), shp, dtype)
        Y, hist = fit_mpo_mps(O, X, opts, init, dtype)
        if counts is not None:
            counts.append(len(hist))
        nrm = float(np.linalg.norm(Y[0]))
        if not np.isfinite(nrm) or nrm == 0.0:
            raise FloatingPointError("column MPS vanished")
        Y[0] = Y[0] / nrm
        X = Y
        kept[c] = X
        if warm is not None:
            warm[c] = [s.copy() for s in Y]
    return kept if keep else X


def extract_message(X):
    """Drop the two corner sites (both 1x1x1 after the last column) into the message. (Eq. 1: the outgoing message is what is left after the last column, App. A.)"""
    assert X[0].shape == (1, 1, 1) and X[-1].shape == (1, 1, 1)
    M = [s.copy() for s in X[1:-1]]
    M[0] = M[0] * X[0][0, 0, 0] * X[-1][0, 0, 0]
    return M


# --------------------------------------------------------------------------------------
# Lattice, partition, sweeps (Sec. "The blockBP algorithm", Eq. 1).
# --------------------------------------------------------------------------------------
@dataclass
class Lattice:
    """blockBP problem.

    OBC: Lx columns x Ly rows, tensors[r*Lx + c] with edge legs of dimension 1.
    INFINITE: Lx x Ly is the unit cell; the single block (by x bx, multiples of the
    cell) is tiled from it and messages itself (Sec. "The blockBP algorithm": one
    block suffices for an iPEPS; incoming left = own outgoing right, etc.).
    shift: (sx, sy), the partition shifted by sx columns and sy rows (the paper covers every
    bond from a block centre by several partitions of the lattice into blocks, shifts of one
    another, Sec. "The blockBP algorithm").  INFINITE: block site (r, c) is lattice site
    (r + sy, c + sx).  OBC (0 <= sx < bx, 0 <= sy < by): the block boundaries move to columns
    sx, sx + bx, ... and rows sy, sy + by, ..., so the blocks on the lattice edges are
    narrower.  The paper embeds the OBC lattice in a periodic one and shifts that; a block
    straddling the embedding's seam is two pieces joined only by bonds of dimension 1, across
    which every message and environment factorises, so it acts as the two edge blocks here.
    single_layer: the tensors are the network's own site tensors E[u, l, d, r] with
    bond D on every leg (d = 1, real; a 2D classical model's partition function, Sec.
    on the 2D Ising model), used as they are instead of a double layer; a term's
    "operator" at a site is then the impurity tensor that replaces E there.
    hermitian_basis: run the whole method after the fixed unitary change of basis of
    hermitian_basis_matrix on every merged leg (not a step of the paper; the basis in which
    the double layer and the messages of a complex PEPS are real).  Every contraction keeps
    its value, so only the arithmetic changes: real E, real messages and real fits (drawn as
    real numbers); E^O of a read-out term is that of the complex double layer, transformed.
    fit_sweeps: per message sweep, the number of fit sweeps every column fit ran (App. A stop
    rule), summed over the messages.
    readout_fit_tol: the fit tolerance of the read-out's environment fits (None: fit_tol).
    """
    Lx: int
    Ly: int
    d: int
    D: int
    bx: int
    by: int
    tensors: list
    boundary: str = "obc"
    chi: int = 16
    chi_exp: int = 0
    fit_tol: float = 1e-6
    fit_max_sweeps: int = 10
    seed: int = 0
    init_mode: int = 0
    warm_start: int = 0  # 0 cold; 1 sweeps warm-started; 2 also the read-out (reading 8)
    single_layer: bool = False
    shift: tuple = (0, 0)
    hermitian_basis: bool = False
    readout_fit_tol: float | None = None
    msgs: dict = field(default_factory=dict)
    warm: dict = field(default_factory=dict)
    sweeps_done: int = 0
    residuals: list = field(default_factory=list)
    fit_sweeps: list = field(default_factory=list)

    def __post_init__(self):
        """The partition into blocks, the double layers (Fig. 1(a,b)) and the initial messages
        (App. A)."""
        assert self.boundary in ("obc", "infinite")
        sx, sy = self.shift
        if self.boundary == "obc":
            assert self.Lx % self.bx == 0 and self.Ly % self.by == 0
            assert 0 <= sx < self.bx and 0 <= sy < self.by
            assert len(self.tensors) == self.Lx * self.Ly
            # block boundaries: every bx columns from sx (every by rows from sy)
            self.xs = sorted({0, self.Lx} | set(range(sx, self.Lx, self.bx)))
            self.ys = sorted({0, self.Ly} | set(range(sy, self.Ly, self.by)))
        else:
            assert self.bx % self.Lx == 0 and self.by % self.Ly == 0
            assert 0 <= sx < self.Lx and 0 <= sy < self.Ly
            assert len(self.tensors) == self.Lx * self.Ly
            self.xs, self.ys = [0, self.bx], [0, self.by]
        self.nbx, self.nby = len(self.xs) - 1, len(self.ys) - 1
        # bond of the double-layer (or single-layer) network; the read-out bond of App. A,
        # 2D^2 + 10, is 2K + 10 in these terms
        self.K = self.D if self.single_layer else self.D * self.D
        if self.chi_exp <= 0:
            self.chi_exp = max(self.chi, 2 * self.K + 10)
        cplx = any(np.iscomplexobj(t) for t in self.tensors)
        self.dtype = np.complex128 if cplx else np.float64
        hb = self.hermitian_basis
        assert not (hb and self.single_layer), "a single-layer network has no (ket, bra) legs"
        if self.single_layer:
            assert self.d == 1 and not cplx, "a single-layer network is real and has no physical leg"
            self.tensors = [np.asarray(t, dtype=np.float64).reshape(np.shape(t)[-4:]) for t in self.tensors]
            self.E = list(self.tensors)
        else:
            self.tensors = [np.asarray(t, dtype=self.dtype) for t in self.tensors]
            self.E = [double_layer(t) for t in self.tensors]
        if hb:
            self.E = [np.ascontiguousarray(to_hermitian_basis_E(e, t.shape[1:]).real)
                      for e, t in zip(self.E, self.tensors)]
            self.dtype = np.float64
        for bi in range(self.nbx * self.nby):
            for dr in self.directions(bi):
                n = self.edge_length(bi, dr)
                stream = stream_id(2, 0, 4 * bi + dr, 0, 0)
                if self.single_layer:
                    m = ones_message(n, self.K, self.dtype) if self.init_mode == 0 else \
                        uniform_message(n, self.K, self.seed, stream, self.dtype)
                elif self.init_mode == 0:
                    m = identity_message(n, self.D, self.dtype)
                else:
                    m = random_mpdo_message(n, self.D, self.seed, stream, self.dtype)
                if hb:
                    # a message carries the legs of the side it leaves through: right and down
                    # legs are in the conj(V) basis
                    m = [np.ascontiguousarray(x.real) for x in
                         to_hermitian_basis_mps(m, self.D, conj_basis=dr in (RIGHT, DOWN))]
                self.msgs[(bi, dr)] = embed_at_caps(normalise_message(m, self.D, self.single_layer), self.chi)

    # -- geometry ------------------------------------------------------------------
    def tensor_index(self, r, c):
        """Site (r, c) -> index into tensors (OBC: r*Lx+c; INFINITE: unit cell). (Sec. "The blockBP algorithm": partition of the lattice into blocks.)"""
        if self.boundary == "obc":
            return r * self.Lx + c
        sx, sy = self.shift
        return ((r + sy) % self.Ly) * self.Lx + ((c + sx) % self.Lx)

    def block_origin(self, bi):
        """(row, column) of block bi's top-left site (Sec. "The blockBP algorithm")."""
        R, C = divmod(bi, self.nbx)
        return self.ys[R], self.xs[C]

    def block_size(self, bi):
        """(rows, columns) of block bi. (Sec. "The blockBP algorithm"; a shifted OBC partition has narrower blocks on the lattice edges.)"""
        R, C = divmod(bi, self.nbx)
        return self.ys[R + 1] - self.ys[R], self.xs[C + 1] - self.xs[C]

    def edge_length(self, bi, dr):
        """Sites along side dr of block bi (the length of a message through it). (Sec. "The blockBP algorithm": a message is an MPS along the shared block edge.)"""
        h, w = self.block_size(bi)
        return h if dr in (LEFT, RIGHT) else w

    def block_of(self, r, c):
        """Block containing lattice site (r, c) (OBC). (Sec. "The blockBP algorithm".)"""
        R = max(i for i in range(self.nby) if self.ys[i] <= r)
        C = max(i for i in range(self.nbx) if self.xs[i] <= c)
        return R * self.nbx + C

    def neighbour(self, bi, dr):
        """Block on side dr of block bi, or None at an OBC lattice edge. (Sec. "The blockBP algorithm": the block graph.)"""
        if self.boundary == "infinite":
            return bi
        R, C = divmod(bi, self.nbx)
        R2, C2 = R + {UP: -1, DOWN: 1}.get(dr, 0), C + {LEFT: -1, RIGHT: 1}.get(dr, 0)
        if 0 <= R2 < self.nby and 0 <= C2 < self.nbx:
            return R2 * self.nbx + C2
        return None

    def directions(self, bi):
        """Outgoing directions whose receiver exists (interior edges; all four if infinite). (Sec. "The blockBP algorithm".)"""
        return [dr for dr in (LEFT, RIGHT, UP, DOWN) if self.neighbour(bi, dr) is not None]

    def block_E(self, bi, ops=None):
        """Double layers of block bi's sites (Fig. 1(a,b)), E^O at the sites in ops."""
        r0, c0 = self.block_origin(bi)
        h, w = self.block_size(bi)
        ops = ops or {}
        grid = []
        for r in range(h):
            row = []
            for c in range(w):
                t = self.tensor_index(r0 + r, c0 + c)
                row.append(self.site_operator(t, ops[(r, c)]) if (r, c) in ops else self.E[t])
            grid.append(row)
        return grid

    def site_operator(self, t, op):
        """E^O of tensor t: the double layer with op on the ket (Fig. 1(a,b)), or, on a
        single-layer network, the impurity tensor op itself."""
        if self.single_layer:
            op = np.asarray(op, dtype=np.float64)
            assert op.shape == self.E[t].shape, "an impurity tensor has the shape of the site tensor it replaces"
            return op
        EO = double_layer(self.tensors[t], op)
        if self.hermitian_basis:
            EO = to_hermitian_basis_E(EO, self.tensors[t].shape[1:])
        return EO

    def incoming(self, bi, msgs=None):
        """Messages into block bi: the neighbour's outgoing message toward bi, or the
        trivial message at an OBC edge. (Eq. 1: the messages a block receives; App. A, OBC edges.)"""
        msgs = self.msgs if msgs is None else msgs
        out = {}
        for dr in (LEFT, RIGHT, UP, DOWN):
            nb = self.neighbour(bi, dr)
            n = self.edge_length(bi, dr)
            out[dr] = trivial_mps(n, self.dtype) if nb is None else msgs[(nb, OPPOSITE[dr])]
        return out

    # -- Eq. 1 -----------------------------------------------------------------------
    def compute_message(self, bi, dr, msgs, sweep_index, counts=None):
        """m_{A->B}^{(l+1)} = Tr(T_A prod_{A' in N_A minus B} m_{A'->A}^{(l)}) (Eq. 1)."""
        Ef, mT, mR, mB = frame(self.block_E(bi), self.incoming(bi, msgs), dr)
        opts = FitOpts(self.chi, self.fit_tol, self.fit_max_sweeps)
        msg = 4 * bi + dr
        warm = self.warm.setdefault((bi, dr), {}) if self.warm_start else None
        X = column_sweep(Ef, mT, mR, mB, opts, self.seed,
                         lambda c, i: stream_id(0, sweep_index, msg, c, i), self.dtype, warm=warm, counts=counts)
        return normalise_message(extract_message(X), self.D, self.single_layer)

    def sweep(self):
        """One synchronous (Jacobi) update of every message; returns the residual
        r = mean over messages of ||m_new - m_old||^2 = mean(2 - 2 Re<m_new|m_old>). (Eq. 1, synchronous update; the residual is the mean squared distance of the unit-norm, phase-fixed messages.)"""
        old = self.msgs
        new = {}
        counts = []
        for (bi, dr) in old:
            new[(bi, dr)] = self.compute_message(bi, dr, old, self.sweeps_done, counts)
        self.fit_sweeps.append(int(sum(counts)))
        res = float(np.mean([2.0 - 2.0 * mps_overlap(new[k], old[k]).real for k in old])) if old else 0.0
        self.msgs = new
        self.sweeps_done += 1
        self.residuals.append(res)
        return res

    def run(self, n_sweeps=0, tol=1e-5, max_sweeps=10, relative=False):
        """Iterate Eq. 1.  n_sweeps > 0: exactly that many; else until the residual
        (absolute, Sec. "The blockBP algorithm"; or relative r_l / r_1, App. A) is below
        tol or max_sweeps is reached.  Returns (residual, sweeps, converged)."""
        if n_sweeps > 0:
            r = 0.0
            for _ in range(n_sweeps):
                r = self.sweep()
            return r, n_sweeps, True
        r1 = None
        r = float("inf")
        for k in range(max_sweeps):
            r = self.sweep()
            r1 = r if r1 is None else r1
            crit = (r / r1 if r1 > 0 else 0.0) if relative else r
            if crit < tol:
                return r, k + 1, True
        return r, max_sweeps, False

    # -- read-out (App. A, Fig. 1(f)) -----------------------------------------------------
    def region_for(self, sites):
        """Block region for terms inside one block; merged two-block region for a
        nearest-neighbour pair across a block edge (reading taken where the paper uses
        shifted partitions instead).  Returns (region id, r0, c0, h, w, blocks)."""
        rc = [divmod(s, self.Lx if self.boundary == "obc" else self.bx) for s in sites]
        if self.boundary == "infinite":
            for r, c in rc:
                if not (0 <= r < self.by and 0 <= c < self.bx):
                    raise ValueError("site outside the block")
            return 0, 0, 0, self.by, self.bx, [0]
        blks = []
        for r, c in rc:
            if not (0 <= r < self.Ly and 0 <= c < self.Lx):
                raise ValueError("site outside the lattice")
            blks.append(self.block_of(r, c))
        nb = self.nbx * self.nby
        if len(set(blks)) == 1:
            bi = blks[0]
            r0, c0 = self.block_origin(bi)
            h, w = self.block_size(bi)
            return bi, r0, c0, h, w, [bi]
        (r1, c1), (r2, c2) = rc
        if abs(r1 - r2) + abs(c1 - c2) != 1:
            raise ValueError("two-site term across blocks must be nearest neighbours")
        a, b = sorted(blks)
        r0, c0 = self.block_origin(a)
        (ha, wa), (hb, wb) = self.block_size(a), self.block_size(b)
        if c1 != c2:  # horizontal pair: a left of b
            return nb + 2 * a, r0, c0, ha, wa + wb, [a, b]
        return nb + 2 * a + 1, r0, c0, ha + hb, wa, [a, b]

    def region_incoming(self, blocks, horizontal):
        """Incoming messages of a block or a merged two-block region.  The two messages
        on a long side of a merged region are joined with a bond of dimension 1, since
        the blockBP environment has no bond between different blocks' messages."""
        if len(blocks) == 1:
            return self.incoming(blocks[0])
        ia, ib = self.incoming(blocks[0]), self.incoming(blocks[1])
        if horizontal:
            return {LEFT: ia[LEFT], RIGHT: ib[RIGHT], UP: ia[UP] + ib[UP], DOWN: ia[DOWN] + ib[DOWN]}
        return {UP: ia[UP], DOWN: ib[DOWN], LEFT: ia[LEFT] + ib[LEFT], RIGHT: ia[RIGHT] + ib[RIGHT]}

    def region_envs(self, rid, r0, c0, h, w, blocks):
        """Column environments with bond chi_exp (App. A uses chi = 2D^2+10 here):
        Lenv[c] = left edge absorbed up to column c-1, Renv[c] = right edge absorbed
        down to column c+1."""
        grid = [[self.E[self.tensor_index(r0 + r, c0 + c)] for c in range(w)] for r in range(h)]
        horizontal = len(blocks) == 2 and blocks[0] // self.nbx == blocks[1] // self.nbx
        m_in = self.region_incoming(blocks, horizontal=horizontal)
        tol = self.fit_tol if self.readout_fit_tol is None else self.readout_fit_tol
        opts = FitOpts(self.chi_exp, tol, self.fit_max_sweeps)
        # Warm read-out (option warm_start = 2, reading 8): with chi_exp = chi, the environment
        # columns of a one-block region in the LEFT (RIGHT) frame are the fits the sweep runs for
        # that block's LEFT (RIGHT) message; each column's fit starts from a copy of the sweep's
        # last one.
        warm = {LEFT: None, RIGHT: None}
        if self.warm_start == 2 and self.chi_exp == self.chi and len(blocks) == 1:
            for dr in (LEFT, RIGHT):
                warm[dr] = {c: [x.copy() for x in Y] for c, Y in self.warm.get((blocks[0], dr), {}).items()}
        Ef, mT, mR, mB = frame(grid, m_in, LEFT)
        keptR = column_sweep(Ef, mT, mR, mB, opts, self.seed,
                             lambda c, i: stream_id(1, rid, 0, c, i), self.dtype, keep=True, warm=warm[LEFT])
        Ef, mT, mR, mB = frame(grid, m_in, RIGHT)
        keptL = column_sweep(Ef, mT, mR, mB, opts, self.seed,
                             lambda c, i: stream_id(1, rid, 1, c, i), self.dtype, keep=True, warm=warm[RIGHT])
        Renv = {c: keptR[c + 1] for c in range(w)}
        Lenv = {c: keptL[w - c] for c in range(w)}
        return grid, m_in, Lenv, Renv

    def expect(self, terms):
        """<O> = N_O / N_I for each term (list of [(site, op), ...] with 1 or 2 sites).

        The closing contraction runs exactly from top to bottom through
        Lenv[c] . column c (. column c+1) . Renv[c or c+1], with E^O at the operator
        sites, and the ratio is taken in FP64 / complex128.
        (App. A read-out, Fig. 1(f).)
        """
        cache = {}
        out = []
        for term in terms:
            sites = [s for s, _ in term]
            reg = self.region_for(sites)
            rid, r0, c0, h, w, blocks = reg
            if rid not in cache:
                cache[rid] = self.region_envs(*reg)
            grid, m_in, Lenv, Renv = cache[rid]
            W = self.Lx if self.boundary == "obc" else self.bx
            loc = {}
            for s, op in term:
                r, c = divmod(s, W)
                loc[(r - r0, c - c0)] = op
            cols = sorted({c for _, c in loc})
            if len(cols) == 2 and cols[1] != cols[0] + 1:
                raise ValueError("two-site term must lie in one column or two adjacent columns")
            cs = list(range(cols[0], cols[-1] + 1))
            num = self._close(grid, m_in, Lenv, Renv, r0, c0, cs, loc)
            den = self._close(grid, m_in, Lenv, Renv, r0, c0, cs, {})
            out.append(num / den)
        return np.array(out, dtype=np.complex128)

    def rdm(self, sites):
        """Reduced density matrix of 1 or 2 sites (the 2-local RDMs the paper compares
        between methods, Sec. on the transverse Ising model): rho = Tr_rest |psi><psi| /
        <psi|psi>, indices (site0, site1) row-major.  Entry (a, b) is <a|rho|b> = Tr(rho |b><a|),
        read out as the expectation of the matrix unit |b><a| (a product of single-site units
        for two sites), so that Tr(rho O) = <O>."""
        assert not self.single_layer, "a single-layer network has no physical leg"
        d, n = self.d, len(sites)
        dim = d ** n
        terms = []
        for a in range(dim):
            for b in range(dim):
                ai, bi = np.unravel_index(a, (d,) * n), np.unravel_index(b, (d,) * n)
                term = []
                for k, s in enumerate(sites):
                    U = np.zeros((d, d))
                    U[bi[k], ai[k]] = 1.0
                    term.append((s, U))
                terms.append(term)
        return self.expect(terms).reshape(dim, dim)

    def _close(self, grid, m_in, Lenv, Renv, r0, c0, cs, loc):
        """Exact top-to-bottom transfer through Lenv[cs[0]], columns cs, Renv[cs[-1]]. (App. A read-out: the exact closing of the region.)"""
        L, R = Lenv[cs[0]], Renv[cs[-1]]
        h = len(grid)
        mT, mB = m_in[UP], m_in[DOWN]
        # rows of MPO tensors per column, all as O[u, l, d, r] (vertical in/out, horizontal in/out)
        colops = []
        for c in cs:
            col = [mT[c][None]]  # [1, alpha_c, v, alpha_{c+1}] as u,l,d,r
            for r in range(h):
                if (r, c) in loc:
                    col.append(self.site_operator(self.tensor_index(r0 + r, c0 + c), loc[(r, c)]))
                else:
                    col.append(grid[r][c])
            col.append(mB[c].transpose(1, 0, 2)[:, :, None, :])  # [v, beta_c, 1, beta_{c+1}]
            colops.append(col)
        # Row transfer F[a, w.., b] -> F'[A, v.., B], one tensor at a time.
        if len(cs) == 1:
            F = np.ones((1, 1, 1), dtype=np.complex128)
            for i in range(h + 2):
                G = np.tensordot(F, L[i], axes=([0], [0]))               # [w, b, s, A]
                G = np.tensordot(G, colops[0][i], axes=([0, 2], [0, 1]))  # [b, A, v, t]
                F = np.tensordot(G, R[i], axes=([0, 3], [0, 1]))          # [A, v, B]
            return F[0, 0, 0]
        F = np.ones((1, 1, 1, 1), dtype=np.complex128)
        for i in range(h + 2):
            G = np.tensordot(F, L[i], axes=([0], [0]))                   # [w, z, b, s, A]
            G = np.tensordot(G, colops[0][i], axes=([0, 3], [0, 1]))      # [z, b, A, v, m]
            G = np.tensordot(G, colops[1][i], axes=([0, 4], [0, 1]))      # [b, A, v, y, t]
            F = np.tensordot(G, R[i], axes=([0, 4], [0, 1]))              # [A, v, y, B]
        return F[0, 0, 0, 0]


def trace_distance(rho, sigma):
    """D(rho, sigma) = (1/2) ||rho - sigma||_1 (the paper's RDM comparison, Sec. on the
    transverse Ising model): half the sum of |eigenvalues| of the Hermitian difference."""
    diff = np.asarray(rho) - np.asarray(sigma)
    return 0.5 * float(np.sum(np.abs(np.linalg.eigvalsh(0.5 * (diff + np.conj(diff.T))))))
