"""MPO of the vibronic Hamiltonian (Eq. MPO) - oracle side.

Test infrastructure only (see the package docstring).

Construction: a finite-state automaton over the chain. At every bond each
term is in one of three kinds of state: 'start' (none of its operators placed
yet), 'done' (all placed) or an open state keyed by the exact tuple of
(position, operator) already placed. Terms that share a prefix share the open
state. The coefficient is applied with the last operator of each term, so
transitions into 'done' are summed over terms and all other transitions are
plain (coefficient-free) operators.

Tensor layout: W[p][w_in, s_out, s_in, w_out], i.e. the operator is
sum W^{s_out, s_in}_{w_in, w_out} |s_out><s_in| as in Eq. MPO.
"""
from __future__ import annotations

import numpy as np

from vibmodels import local_dims
from .vibronic import local_matrix, term_list

START = ("start",)
DONE = ("done",)


def _key(sorted_ops, b):
    """State of a term at bond b (between positions b and b+1)."""
    first = sorted_ops[0][0]
    last = sorted_ops[-1][0]
    if last <= b:
        return DONE
    if first > b:
        return START
    return tuple(o for o in sorted_ops if o[0] <= b)


def build_mpo(model: dict):
    """Returns the list of site tensors W[p] (float64)."""
    dims = local_dims(model)
    n = len(dims)
    terms = []
    for coef, ops in term_list(model):
        terms.append((coef, sorted(ops.items())))
    # channel sets per bond: bond -1 = {START}, bond n-1 = {DONE}
    chans = []
    for b in range(-1, n):
        ks = set()
        for _, so in terms:
            ks.add(_key(so, b))
        if b == -1:
            ks = {START}
        if b == n - 1:
            ks = {DONE}
        rest = sorted(k for k in ks if k not in (START, DONE))
        ordered = [k for k in (START, DONE) if k in ks] + rest
        chans.append({k: idx for idx, k in enumerate(ordered)})
    W = []
    for p in range(n):
        cin, cout = chans[p], chans[p + 1]
        d = dims[p]
        Wp = np.zeros((len(cin), d, d, len(cout)))
        fixed = {}
        for coef, so in terms:
            kin = _key(so, p - 1)
            kout = _key(so, p)
            ops_here = [o for (q, o) in so if q == p]
            if ops_here:
                mat = local_matrix(model, p, ops_here[0])
            else:
                mat = np.eye(d)
            if kout == DONE and kin != DONE:
                Wp[cin[kin], :, :, cout[kout]] += coef * mat
            else:
                key = (cin[kin], cout[kout])
                if key in fixed:
                    assert np.array_equal(fixed[key], mat)
                else:
                    fixed[key] = mat
        if p > 0 and DONE in cin and DONE in cout:
            fixed[(cin[DONE], cout[DONE])] = np.eye(d)
        for (i, o), mat in fixed.items():
            Wp[i, :, :, o] = mat
        W.append(Wp)
    return W


def mpo_to_dense(W) -> np.ndarray:
    """Contract the MPO into the full operator (tiny systems only)."""
    acc = W[0][0]  # [O, I, w]: the single left boundary channel dropped
    for Wp in W[1:]:
        # acc[O, I, w] Wp[w, o, i, v] -> [O o, I i, v]
        t = np.einsum("OIw,woiv->OoIiv", acc, Wp)
        O, o, I, i, v = t.shape
        acc = t.reshape(O * o, I * i, v)
    return acc[:, :, 0]


def mpo_bond_dims(W):
    return [Wp.shape[3] for Wp in W[:-1]]
