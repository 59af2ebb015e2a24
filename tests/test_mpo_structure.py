"""Why the MPO is the exact finite-state-automaton construction with no
compression tolerance: an SVD compression of the vibronic MPO lowers its bond
dimension, but it mixes the channels, so the automaton's few nonzero blocks
(mostly exact identities, the rest banded operators q, q^2, n and their sums)
become fully populated banded blocks with no identities left, many times
more work for the sparse H_eff legs than the dense legs save. These CPU tests
pin those facts on the bench workload and check the compression itself
against the dense Hamiltonian on a small model."""
import numpy as np

import vibmodels as vm
from oracle import mpo as ompo


def _svd_compress(W, tol=1e-12):
    """Left-to-right QR, right-to-left SVD truncation at tol of the largest
    singular value of each bond; returns the compressed site tensors
    (w_l, d, d, w_r) and their bond dimensions."""
    W = [np.array(w, dtype=float) for w in W]
    n = len(W)
    for p in range(n - 1):
        wl, d1, d2, wr = W[p].shape
        q, r = np.linalg.qr(W[p].reshape(wl * d1 * d2, wr))
        W[p] = q.reshape(wl, d1, d2, q.shape[1])
        W[p + 1] = np.tensordot(r, W[p + 1], axes=(1, 0))
    for p in range(n - 1, 0, -1):
        wl, d1, d2, wr = W[p].shape
        u, s, vt = np.linalg.svd(W[p].reshape(wl, d1 * d2 * wr), full_matrices=False)
        k = int(np.sum(s > tol * s[0]))
        W[p] = vt[:k].reshape(k, d1, d2, wr)
        W[p - 1] = np.tensordot(W[p - 1], u[:, :k] * s[:k], axes=(3, 0))
    return W, [w.shape[3] for w in W[:-1]]


def _block_kinds(W):
    """Counts of (w_in, w_out) blocks of the site tensors: zero, multiples of
    the identity, banded with bandwidth <= 2, and dense otherwise."""
    zero = ident = banded = dense = 0
    for w in W:
        d = w.shape[1]
        off = np.abs(np.subtract.outer(np.arange(d), np.arange(d)))
        for a in range(w.shape[0]):
            for b in range(w.shape[3]):
                blk = w[a, :, :, b]
                mx = np.max(np.abs(blk))
                if mx <= 1e-12:
                    zero += 1
                elif np.allclose(blk, blk[0, 0] * np.eye(d), atol=1e-12 * mx):
                    ident += 1
                elif np.max(np.abs(blk[off > 2]), initial=0.0) <= 1e-12 * mx:
                    banded += 1
                else:
                    dense += 1
    return zero, ident, banded, dense


def test_svd_compression_is_exact_on_a_small_model():
    m = vm.model_small_2state(n_modes=3, levels=4)
    W = ompo.build_mpo(m)
    Wc, bonds = _svd_compress(W)
    h, hc = ompo.mpo_to_dense(W), ompo.mpo_to_dense(Wc)
    assert np.max(np.abs(h - hc)) <= 1e-12 * np.max(np.abs(h))
    assert all(b <= a for a, b in zip(ompo.mpo_bond_dims(W)[1:-1], bonds))


def test_compression_halves_the_bond_but_fills_every_block():
    m = vm.model_internal_conversion()
    W = ompo.build_mpo(m)
    fsa = [w.shape[3] for w in W[:-1]]
    Wc, bonds = _svd_compress(W)
    # the compression roughly halves the bond dimension of the bench workload
    assert max(fsa) == 26 and max(bonds) == 14
    # ... but the automaton's nonzero blocks are mostly identities (an add per
    # element in the sparse legs) and few banded operators, while every block
    # of the compressed tensors is a banded combination of them
    z, i, b, d = _block_kinds(W)
    assert d == 0 and i > 2 * b > 0
    zc, ic, bc, dc = _block_kinds(Wc)
    assert zc == 0 and ic == 0 and dc == 0 and bc > 4 * (i + b)
    # sparse-leg work with ~2 flop per element for an identity block and ~20
    # for a banded one (5 diagonals, real x complex): over ten times more
    assert 20 * bc > 10 * (2 * i + 20 * b)
