"""Independent exact references used to pin the oracle (test helpers only).

Nothing here shares code with ``oracle/`` or with the CUDA library:

* ``state_vector``: the PEPS amplitude vector by direct contraction of the
  single-layer network, site by site (no double layer, no messages, no fits).
* ``exact_expect``: <psi|O|psi>/<psi|psi> from that vector.
* ``textbook_bp``: plain belief propagation on the double-layer network with one
  site per node (the method blockBP reduces to for blocks of size 1, Sec. "The
  blockBP algorithm"), written as vector messages on lattice edges.
* ``dense_mps`` / ``dense_mpo_apply``: dense vectors of small MPS and of O|X>.
"""
from __future__ import annotations

import numpy as np


def state_vector(tensors, Lx, Ly):
    """Amplitudes psi[p_0, ..., p_{N-1}] of an OBC PEPS (row-major site order)."""
    d = tensors[0].shape[0]
    dt = np.result_type(*tensors)
    # S axes: (phys so far), frontier vertical legs for each column, horizontal leg
    S = np.ones((1,) + (1,) * Lx + (1,), dtype=dt)
    for r in range(Ly):
        for c in range(Lx):
            T = tensors[r * Lx + c]  # p,u,l,d,r
            nd = S.ndim
            # axes of S: 0 = phys, 1..Lx = frontier, Lx+1 = horizontal
            fr = 1 + c
            S = np.tensordot(S, T, axes=([fr, nd - 1], [1, 2]))
            # S now: phys, frontier(without c), p, d, r  -> reorder
            axes = list(range(S.ndim))
            phys_new, dnew, rnew = S.ndim - 4 + 1, S.ndim - 2, S.ndim - 1
            p_ax = S.ndim - 3
            rest = [a for a in axes if a not in (0, p_ax, dnew, rnew)]
            order = [0, p_ax] + rest[:c] + [dnew] + rest[c:] + [rnew]
            S = S.transpose(order)
            shp = S.shape
            S = S.reshape((shp[0] * shp[1],) + shp[2:])
    return S.reshape(-1)


def exact_expect(psi, n_sites, d, term):
    """<psi| prod_k O_k |psi> / <psi|psi> for term = [(site, O), ...]."""
    phi = psi.reshape((d,) * n_sites).astype(np.complex128)
    for s, O in term:
        phi = np.moveaxis(np.tensordot(O, phi, axes=([1], [s])), 0, s)
    return np.vdot(psi, phi.reshape(-1)) / np.vdot(psi, psi)


def _dl(T, O=None):
    """Double-layer tensor of one site (written independently of the oracle)."""
    d = T.shape[0]
    Dshape = T.shape[1:]
    ket = T if O is None else np.tensordot(O, T, axes=([1], [0]))
    E = np.zeros(tuple(x * x for x in Dshape), dtype=np.complex128)
    for p in range(d):
        E += _kron4(ket[p], np.conj(T[p]))
    return E


def _kron4(a, b):
    """E[(u u'),(l l'),(d d'),(r r')] = a[u,l,d,r] b[u',l',d',r']."""
    o = np.multiply.outer(a, b)  # u l d r u' l' d' r'
    o = o.transpose(0, 4, 1, 5, 2, 6, 3, 7)
    s = o.shape
    return o.reshape(s[0] * s[1], s[2] * s[3], s[4] * s[5], s[6] * s[7])


def textbook_bp(tensors, Lx, Ly, terms, iters=200, tol=1e-14, boundary="obc"):
    """Site-level BP on the double-layer network.

    m[(i, dir)] is the vector message sent by site i toward its neighbour in
    direction dir (0 left, 1 right, 2 up, 3 down), of the dimension of that leg.
    Update: contract E_i with the incoming messages on its other legs; normalise to
    unit 2-norm.  Read-out: 1-site <O> = Tr(E^O prod m) / Tr(E prod m); a nearest-
    neighbour pair contracts both sites' tensors over their shared leg.
    """
    N = Lx * Ly
    E = [_dl(t) for t in tensors]
    leg = {0: 1, 1: 3, 2: 0, 3: 2}  # dir -> axis of E[u,l,d,r]

    def nbr(i, dr):
        r, c = divmod(i, Lx)
        r2, c2 = r + {2: -1, 3: 1}.get(dr, 0), c + {0: -1, 1: 1}.get(dr, 0)
        if boundary == "obc":
            if 0 <= r2 < Ly and 0 <= c2 < Lx:
                return r2 * Lx + c2
            return None
        return (r2 % Ly) * Lx + (c2 % Lx)

    opp = {0: 1, 1: 0, 2: 3, 3: 2}
    m = {}
    for i in range(N):
        for dr in range(4):
            if nbr(i, dr) is not None:
                dim = E[i].shape[leg[dr]]
                D = int(round(np.sqrt(dim)))
                m[(i, dr)] = np.eye(D).reshape(-1).astype(np.complex128)

    def incoming(i, dr):
        j = nbr(i, dr)
        if j is None:
            return np.ones(1, dtype=np.complex128)
        return m[(j, opp[dr])]

    def contract_except(Ei, i, skip):
        t = Ei
        # contract legs in decreasing axis order so remaining axis numbers stay valid
        for dr in sorted([x for x in range(4) if x != skip], key=lambda x: -leg[x]):
            t = np.tensordot(t, incoming(i, dr), axes=([leg[dr]], [0]))
        return t

    for _ in range(iters):
        new = {}
        for (i, dr) in m:
            v = contract_except(E[i], i, dr)
            new[(i, dr)] = v / np.linalg.norm(v)
        delta = max(np.linalg.norm(new[k] - m[k]) for k in m)
        m = new
        if delta < tol:
            break

    def full(Ei, i):
        t = Ei
        for dr in sorted(range(4), key=lambda x: -leg[x]):
            t = np.tensordot(t, incoming(i, dr), axes=([leg[dr]], [0]))
        return t

    out = []
    for term in terms:
        if len(term) == 1:
            (s, O), = term
            out.append(full(_dl(tensors[s], O), s) / full(E[s], s))
            continue
        (s1, O1), (s2, O2) = term
        if s2 < s1:
            (s1, O1), (s2, O2) = (s2, O2), (s1, O1)
        dr = 1 if s2 == nbr(s1, 1) else 3
        num = _pair(_dl(tensors[s1], O1), _dl(tensors[s2], O2), s1, s2, dr, incoming, leg, opp)
        den = _pair(E[s1], E[s2], s1, s2, dr, incoming, leg, opp)
        out.append(num / den)
    return np.array(out)


def _pair(E1, E2, s1, s2, dr, incoming, leg, opp):
    t1 = E1
    for x in sorted([x for x in range(4) if x != dr], key=lambda x: -leg[x]):
        t1 = np.tensordot(t1, incoming(s1, x), axes=([leg[x]], [0]))
    t2 = E2
    for x in sorted([x for x in range(4) if x != opp[dr]], key=lambda x: -leg[x]):
        t2 = np.tensordot(t2, incoming(s2, x), axes=([leg[x]], [0]))
    return np.dot(t1, t2)


def dense_mps(M):
    """Dense vector of an open MPS (bond dims 1 at both ends)."""
    v = M[0]
    for s in M[1:]:
        v = np.tensordot(v, s, axes=([-1], [0]))
    return v.reshape(-1)


def dense_mpo_apply(O, X):
    """Dense vector of O|X> for MPO sites O[w,p,q,w'] and MPS sites X[x,p,x']."""
    t = np.ones((1, 1), dtype=np.result_type(O[0], X[0]))  # (w, x) open bonds, phys grown in front
    for o, x in zip(O, X):
        # t: [..., w, x]; contract with x[x,p,x'] and o[w,p,q,w']
        t = np.tensordot(t, x, axes=([-1], [0]))          # [..., w, p, x']
        t = np.tensordot(t, o, axes=([-3, -2], [0, 1]))   # [..., x', q, w']
        t = np.moveaxis(t, -3, -1)                        # [..., q, w', x']
    return t.reshape(-1)


def network_value(E, Lx, Ly, replace=None):
    """Exact contraction of an OBC single-layer network of site tensors E[u, l, d, r]
    (row-major), with E at the sites in `replace` (site -> tensor) swapped for the given
    tensors: a row-by-row transfer over the open vertical legs, no messages, no fits."""
    replace = replace or {}
    # S axes: the open down legs of the previous row, one per column, then the open right leg
    S = np.ones((1,) * Lx + (1,))
    for r in range(Ly):
        for c in range(Lx):
            s = r * Lx + c
            T = np.asarray(replace.get(s, E[s]), dtype=np.float64)
            # contract the column's open leg (axis c) with u and the running right leg with l
            S = np.tensordot(S, T, axes=([c, Lx], [0, 1]))  # axes: other columns..., d, r
            # put the new down leg back at position c; the right leg stays last
            S = np.moveaxis(S, Lx - 1, c)
    return float(S.reshape(-1)[0])


def exact_rdm(psi, n_sites, d, sites):
    """Reduced density matrix of `sites` (index order as given) by the partial trace of
    |psi><psi| / <psi|psi> over every other site."""
    phi = psi.reshape((d,) * n_sites).astype(np.complex128)
    rest = [s for s in range(n_sites) if s not in sites]
    A = np.transpose(phi, list(sites) + rest).reshape(d ** len(sites), -1)
    rho = A @ np.conj(A.T)
    return rho / np.trace(rho)
