"""Seeded synthetic PEPS inputs shared by the tests, the bench and the oracle checks.

This module draws random numbers and lays them out as site tensors; it holds none of
the blockBP arithmetic.  Tensors are numpy arrays T[p, u, l, d, r]; under open
boundaries the legs on the lattice edge have dimension 1.  Sites are drawn in
row-major (r, c) order, each tensor in C order.

The workloads stand in for the ground-state PEPS of the transverse-Ising and
Heisenberg models that the paper studies (those were produced by imaginary-time
evolution and are not available here): positive near-uniform tensors, near-product
tensors, and complex Gaussian unit cells with the same d, D and block shapes.
"""
from __future__ import annotations

import numpy as np

SIGMA_X = np.array([[0.0, 1.0], [1.0, 0.0]])
SIGMA_Y = np.array([[0.0, -1j], [1j, 0.0]])
SIGMA_Z = np.array([[1.0, 0.0], [0.0, -1.0]])


def site_shape(r, c, Lx, Ly, d, D, boundary="obc"):
    """(d, Du, Dl, Dd, Dr) with dimension-1 legs on an open lattice edge."""
    if boundary != "obc":
        return (d, D, D, D, D)
    return (d, 1 if r == 0 else D, 1 if c == 0 else D, 1 if r == Ly - 1 else D, 1 if c == Lx - 1 else D)


def uniform_noise_peps(Lx, Ly, d, D, seed, noise=0.1, boundary="obc", dtype=np.float64):
    """T = U[0,1] + noise * N(0,1): the U block then the N block for each site."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(Ly):
        for c in range(Lx):
            shp = site_shape(r, c, Lx, Ly, d, D, boundary)
            u = rng.random(shp)
            n = rng.standard_normal(shp)
            out.append((u + noise * n).astype(dtype))
    return out


def near_product_peps(Lx, Ly, d, D, seed, noise=0.05, boundary="obc"):
    """One seeded unit vector t (U[0,1]^d normalised) on T[:,0,0,0,0] of every site;
    every entry with a nonzero virtual index is noise * N(0,1)."""
    rng = np.random.default_rng(seed)
    t = rng.random(d)
    t /= np.linalg.norm(t)
    out = []
    for r in range(Ly):
        for c in range(Lx):
            shp = site_shape(r, c, Lx, Ly, d, D, boundary)
            T = noise * rng.standard_normal(shp)
            T[:, 0, 0, 0, 0] = t
            out.append(T)
    return out


def complex_normal_cell(ux, uy, d, D, seed, dtype=np.complex64):
    """Unit cell of ux*uy tensors with real and imaginary parts each N(0,1)/sqrt(D)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(ux * uy):
        shp = (d, D, D, D, D)
        re = rng.standard_normal(shp) / np.sqrt(D)
        im = rng.standard_normal(shp) / np.sqrt(D)
        out.append((re + 1j * im).astype(dtype))
    return out


def product_peps(Lx, Ly, d, D, vecs, boundary="obc"):
    """Product state embedded at bond dimension D: T = t (x) e0 (x) e0 (x) e0 (x) e0."""
    out = []
    for r in range(Ly):
        for c in range(Lx):
            shp = site_shape(r, c, Lx, Ly, d, D, boundary)
            T = np.zeros(shp, dtype=np.result_type(vecs[r * Lx + c], np.float64))
            T[:, 0, 0, 0, 0] = vecs[r * Lx + c]
            out.append(T)
    return out


def gauge_dress(tensors, Lx, Ly, seed, boundary="obc", complex_gauge=False):
    """Insert G G^{-1} on every virtual bond with random well-conditioned G.

    The state is unchanged; the tensors become dense.  On an infinite unit cell the
    bond (r,c)-(r,c+1 mod Lx) and (r,c)-(r+1 mod Ly, c) are dressed consistently.
    """
    rng = np.random.default_rng(seed)
    T = [t.astype(np.complex128 if complex_gauge else np.result_type(t, np.float64)).copy() for t in tensors]

    def rand_gauge(D):
        G = np.eye(D) + 0.3 * rng.standard_normal((D, D))
        if complex_gauge:
            G = G + 0.3j * rng.standard_normal((D, D))
        return G, np.linalg.inv(G)

    for r in range(Ly):
        for c in range(Lx):
            i = r * Lx + c
            # horizontal bond to the right
            if boundary != "obc" or c + 1 < Lx:
                j = r * Lx + (c + 1) % Lx
                D = T[i].shape[4]
                G, Gi = rand_gauge(D)
                T[i] = np.einsum("puldr,rs->pulds", T[i], G)
                T[j] = np.einsum("sr,purdx->pusdx", Gi, T[j])
            # vertical bond downwards
            if boundary != "obc" or r + 1 < Ly:
                j = ((r + 1) % Ly) * Lx + c
                D = T[i].shape[3]
                G, Gi = rand_gauge(D)
                T[i] = np.einsum("puldr,ds->pulsr", T[i], G)
                T[j] = np.einsum("sd,pdlxr->pslxr", Gi, T[j])
    return T


def config(k: int) -> dict:
    """The five benchmark workloads (seed = config number).

    1: 4x4 OBC, d=2, D=2, U[0,1]+0.1N, 2x2 blocks, chi=16, FP64.
    2: 12x12 OBC, d=2, D=3, near-product (+0.05N), 3x3 blocks, chi=32, residual 1e-8; FP32-level
       contractions on TF32 tensor cores (split operands, "tf32x3").
    3: infinite 2x2 cell, d=2, D=4, complex64 N(0,1)/sqrt(D), 4x4 block, chi=64, BF16.
    4: 32x32 OBC, d=2, D=5, U[0,1]+0.1N as float32, 4x4 blocks, chi=96, split-BF16 contractions
       ("bf16x3"), FP64 truncation.
    6: 20x20 OBC, d=2, D=4, U[0,1]+0.1N, 4x4 blocks (80 messages), chi=64, BF16 -- the
       tensor-core measurement workload (D=4, chi=64 contractions over >= 64 messages).
    7: the infinite classical 2D Ising model at beta = 0.6 as its own single-layer network
       (bond 2, 1x1 cell, field 1e-6 selecting the up state), one 8x8 block, chi=32,
       split-TF32 contractions; read out with the magnetisation impurity.
    """
    if k == 1:
        return dict(name="peps4x4_D2_chi16_fp64", Lx=4, Ly=4, d=2, D=2, bx=2, by=2, chi=16,
                    boundary="obc", tensors=uniform_noise_peps(4, 4, 2, 2, seed=1), prec="fp64")
    if k == 2:
        return dict(name="peps12x12_D3_chi32", Lx=12, Ly=12, d=2, D=3, bx=3, by=3, chi=32,
                    boundary="obc", tensors=near_product_peps(12, 12, 2, 3, seed=2), prec="tf32x3",
                    tol=1e-8)
    if k == 3:
        return dict(name="ipeps2x2_D4_chi64_bf16", Lx=2, Ly=2, d=2, D=4, bx=4, by=4, chi=64,
                    boundary="infinite", tensors=complex_normal_cell(2, 2, 2, 4, seed=3), prec="bf16")
    if k == 4:
        # golden: the oracle's values on an 8x8 lattice at the same D, chi and blocks
        return dict(name="peps32x32_D5_chi96", Lx=32, Ly=32, d=2, D=5, bx=4, by=4, chi=96,
                    boundary="obc", tensors=uniform_noise_peps(32, 32, 2, 5, seed=4, dtype=np.float32),
                    prec="bf16x3", golden="d5_chi96_8x8.json")
    if k == 6:
        # tensor-core measurement workload: D=4, chi=64 contractions batched over 80 messages
        return dict(name="peps20x20_D4_chi64_bf16", Lx=20, Ly=20, d=2, D=4, bx=4, by=4, chi=64,
                    boundary="obc", tensors=uniform_noise_peps(20, 20, 2, 4, seed=6), prec="bf16", tol=1e-6)
    if k == 7:
        E, Ez = ising_network(0.6, h=1e-6)
        return dict(name="ising_network_inf_b8_chi32", Lx=1, Ly=1, d=1, D=2, bx=8, by=8, chi=32,
                    boundary="infinite", tensors=[E], impurity=Ez, single_layer=1, prec="tf32x3", tol=1e-8)
    raise ValueError(k)


def standard_terms(Lx, Ly):
    """<sz>, <sx> on every site and <sz sz> on every nearest-neighbour bond (row-major)."""
    terms = []
    for s in range(Lx * Ly):
        terms.append([(s, SIGMA_Z)])
    for s in range(Lx * Ly):
        terms.append([(s, SIGMA_X)])
    for r in range(Ly):
        for c in range(Lx):
            s = r * Lx + c
            if c + 1 < Lx:
                terms.append([(s, SIGMA_Z), (s + 1, SIGMA_Z)])
            if r + 1 < Ly:
                terms.append([(s, SIGMA_Z), (s + Lx, SIGMA_Z)])
    return terms


def ising_peps(beta, h=0.0):
    """One site tensor (1x1 unit cell, d=2, D=2) of the PEPS sum_s exp(beta/2 sum_<ij> s_i s_j) |s>.

    Its norm <psi|psi> is the partition function of the classical 2D Ising model at
    inverse temperature beta, and <psi|sz|psi>/<psi|psi> is that model's magnetisation.
    The bond weight W[s,s'] = exp(beta s s' / 2) is split as W = M M^T (M the symmetric
    square root) and each site carries M[s, .] on its four legs.  h != 0 multiplies the
    amplitudes of up / down by (1 + h) / (1 - h), a small field that selects the up
    ordered state."""
    W = np.array([[np.exp(beta / 2), np.exp(-beta / 2)], [np.exp(-beta / 2), np.exp(beta / 2)]])
    ev, U = np.linalg.eigh(W)
    M = U @ np.diag(np.sqrt(ev)) @ U.T
    T = np.zeros((2, 2, 2, 2, 2))
    for p in range(2):
        T[p] = np.einsum("u,l,d,r->uldr", M[p], M[p], M[p], M[p]) * (1.0 + (h if p == 0 else -h))
    return T


def ising_network(beta, h=0.0):
    """Site tensor E[u, l, d, r] (bond 2) of the single-layer network whose contraction is
    the partition function of the classical 2D Ising model, and the impurity tensor that
    gives sum_s s exp(...) at one site, so that <impurity> = Z_s / Z is the magnetisation.

    The bond weight B[s, s'] = exp(beta s s') (s = +1 for index 0, -1 for index 1) is split
    as B = M M^T (M the symmetric square root) and each site carries M[s, .] on its four
    legs.  h != 0 weights the site's up / down state by (1 + h) / (1 - h), a small field that
    selects the up ordered state."""
    B = np.array([[np.exp(beta), np.exp(-beta)], [np.exp(-beta), np.exp(beta)]])
    ev, U = np.linalg.eigh(B)
    M = U @ np.diag(np.sqrt(ev)) @ U.T
    E = np.zeros((2, 2, 2, 2))
    Ez = np.zeros((2, 2, 2, 2))
    for p, s in ((0, 1.0), (1, -1.0)):
        w = np.einsum("u,l,d,r->uldr", M[p], M[p], M[p], M[p]) * (1.0 + h * s)
        E += w
        Ez += s * w
    return E, Ez


def positive_network(Lx, Ly, K, seed, noise=0.1, boundary="obc"):
    """Single-layer network of real K-leg site tensors E[u, l, d, r] = U[0,1] + noise N(0,1)
    (U block then N block per site, row-major sites, OBC edge legs of dimension 1)."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(Ly):
        for c in range(Lx):
            shp = site_shape(r, c, Lx, Ly, 1, K, boundary)[1:]
            out.append(rng.uniform(0.0, 1.0, shp) + noise * rng.standard_normal(shp))
    return out
