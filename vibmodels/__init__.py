"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws numbers: model parameters of the vibronic Hamiltonian
(Sec. 2.2, Eqs. Hel_2, Hvib_2, Helvib_2) and random dense tensors for kernel
tests. It contains none of the 2TDVP arithmetic, so that the CPU oracle and the
CUDA path can both consume it without sharing any part of the method.

A model is a plain dict:
    n_el        number of electronic states
    e0[n_el]    state energies eps^0_i (eV)
    v0[n_el][n_el]   electronic couplings V^0_ij (eV, symmetric, diagonal ignored)
    omega[n_modes]   mode energies hbar*omega_I (eV)
    levels[n_modes]  local basis size d_I = n_max + 1 (Sec. 2.2, last paragraph)
    g1[n_modes][n_el][n_el]  linear couplings g^I_ij (eV, symmetric in ij)
    g2  list of (I, J, i, j, value): second-order couplings g^{IJ}_ij with
        I <= J; I == J is the quadratic intra-mode term q_I^2, I < J the
        bilinear term q_I q_J. Each entry stands for one operator term; the
        generator adds the (j, i) entry for every off-diagonal (i, j).
    site_order  list over chain positions, -1 = electronic site, k = mode k;
                None = electronic site first, then modes in index order
    include_zpe 1 to include hbar*omega/2 per mode (Eq. Hvib_2)
Units: eV and fs, hbar = 0.6582119569 eV fs.
"""
from __future__ import annotations

import numpy as np

HBAR_EV_FS = 0.6582119569
AU_TIME_FS = 0.02418884326585747


def _empty_model(n_el: int, n_modes: int) -> dict:
    return dict(
        n_el=n_el,
        e0=np.zeros(n_el),
        v0=np.zeros((n_el, n_el)),
        omega=np.zeros(n_modes),
        levels=np.zeros(n_modes, dtype=np.int64),
        g1=np.zeros((n_modes, n_el, n_el)),
        g2=[],
        site_order=None,
        include_zpe=1,
    )


def chain_order(model: dict) -> list:
    """Site order along the chain (-1 = electronic site)."""
    if model.get("site_order") is not None:
        return list(model["site_order"])
    return [-1] + list(range(len(model["omega"])))


def local_dims(model: dict) -> list:
    """Physical dimension of every chain site."""
    out = []
    for s in chain_order(model):
        out.append(int(model["n_el"]) if s < 0 else int(model["levels"][s]))
    return out


def model_small_2state(seed: int = 1001, n_modes: int = 4, levels: int = 8) -> dict:
    """2 states (gap 0.5 eV, coupling 0.1 eV) + n_modes harmonic modes,
    omega ~ U(0.05, 0.2) eV, diagonal linear couplings kappa ~ N(0, 0.05) eV,
    `levels` phonon levels per mode, electronic site first."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = _empty_model(2, n_modes)
    m["e0"] = np.array([-0.25, 0.25])
    m["v0"] = np.array([[0.0, 0.1], [0.1, 0.0]])
    m["omega"] = rng.uniform(0.05, 0.2, n_modes)
    m["levels"] = np.full(n_modes, levels, dtype=np.int64)
    k = rng.normal(0.0, 0.05, (n_modes, 2))
    for I in range(n_modes):
        m["g1"][I, 0, 0] = k[I, 0]
        m["g1"][I, 1, 1] = k[I, 1]
    return m


def model_internal_conversion(seed: int = 1002, n_modes: int = 24,
                              level_range=(10, 30), n_offdiag: int = 6,
                              n_bilinear: int = 24, dense_pairs: bool = False) -> dict:
    """Internal-conversion-like model shaped like the 24-mode pyrazine S1/S2
    Hamiltonian of Sec. 3.1: 2 states (gap 0.5 eV, coupling 0.1 eV), modes with
    omega ~ U(0.05, 0.2) eV and d_I ~ U{level_range}; diagonal linear
    couplings ~ N(0, 0.02); off-diagonal linear g^I_12 ~ N(0, 0.02) on
    `n_offdiag` modes; quadratic intra-mode gamma_II (diagonal in the
    electronic index) ~ N(0, 0.02); bilinear gamma_IJ (diagonal in the
    electronic index) ~ N(0, 0.02) on `n_bilinear` seeded pairs (all pairs
    when dense_pairs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = _empty_model(2, n_modes)
    m["e0"] = np.array([-0.25, 0.25])
    m["v0"] = np.array([[0.0, 0.1], [0.1, 0.0]])
    m["omega"] = rng.uniform(0.05, 0.2, n_modes)
    m["levels"] = rng.integers(level_range[0], level_range[1] + 1, n_modes).astype(np.int64)
    kd = rng.normal(0.0, 0.02, (n_modes, 2))
    for I in range(n_modes):
        m["g1"][I, 0, 0] = kd[I, 0]
        m["g1"][I, 1, 1] = kd[I, 1]
    off_modes = rng.choice(n_modes, size=min(n_offdiag, n_modes), replace=False)
    for I in sorted(off_modes):
        g = rng.normal(0.0, 0.02)
        m["g1"][I, 0, 1] = g
        m["g1"][I, 1, 0] = g
    quad = rng.normal(0.0, 0.02, (n_modes, 2))
    g2 = []
    for I in range(n_modes):
        for i in range(2):
            g2.append((I, I, i, i, float(quad[I, i])))
    if dense_pairs:
        pairs = [(I, J) for I in range(n_modes) for J in range(I + 1, n_modes)]
    else:
        allp = [(I, J) for I in range(n_modes) for J in range(I + 1, n_modes)]
        idx = rng.choice(len(allp), size=min(n_bilinear, len(allp)), replace=False)
        pairs = sorted(allp[k] for k in idx)
    for (I, J) in pairs:
        v = rng.normal(0.0, 0.02, 2)
        for i in range(2):
            g2.append((I, J, i, i, float(v[i])))
    m["g2"] = g2
    return m


def debye_couplings(n_modes: int, lam: float, omega_c: float, omega_max: float):
    """Uniform bath grid omega_I = I*omega_max/n (I = 1..n) and couplings
    g_I = sqrt((2/pi) J(omega_I) d_omega) for the Debye density
    J(w) = 2*lam*w*omega_c/(w^2 + omega_c^2) (Sec. 3.2)."""
    dw = omega_max / n_modes
    w = dw * np.arange(1, n_modes + 1)
    J = 2.0 * lam * w * omega_c / (w * w + omega_c * omega_c)
    g = np.sqrt((2.0 / np.pi) * J * dw)
    return w, g


def model_singlet_fission(seed: int = 1003, n_bath: int = 100, levels: int = 10,
                          lam: float = 0.05, omega_c: float = 0.1,
                          omega_max: float = 0.4) -> dict:
    """Singlet-fission-like model (Sec. 3.2, Table el_SF): states (LE, TT, CT)
    with energies (0.10, 0.00, 0.30) eV, LE-CT and TT-CT couplings
    -U(0.05, 0.1) eV, each state linearly and diagonally coupled to its own
    Debye bath of n_bath modes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_modes = 3 * n_bath
    m = _empty_model(3, n_modes)
    m["e0"] = np.array([0.10, 0.00, 0.30])
    v_le_ct = -rng.uniform(0.05, 0.1)
    v_tt_ct = -rng.uniform(0.05, 0.1)
    v = np.zeros((3, 3))
    v[0, 2] = v[2, 0] = v_le_ct
    v[1, 2] = v[2, 1] = v_tt_ct
    m["v0"] = v
    w, g = debye_couplings(n_bath, lam, omega_c, omega_max)
    for st in range(3):
        for k in range(n_bath):
            I = st * n_bath + k
            m["omega"][I] = w[k]
            m["levels"][I] = levels
            m["g1"][I, st, st] = g[k]
    return m


def model_independent_boson(seed: int = 7, n_el: int = 2, n_modes: int = 3,
                            levels: int = 16, s_max: float = 0.1) -> dict:
    """Displaced-oscillator (independent-boson) model: no electronic coupling,
    diagonal linear couplings chosen so that the Huang-Rhys factor
    S = g^2 / (2 omega^2) lies in [0.02, s_max]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = _empty_model(n_el, n_modes)
    m["e0"] = rng.uniform(-0.3, 0.3, n_el)
    m["omega"] = rng.uniform(0.05, 0.2, n_modes)
    m["levels"] = np.full(n_modes, levels, dtype=np.int64)
    for I in range(n_modes):
        for i in range(n_el):
            S = rng.uniform(0.02, s_max)
            sign = 1.0 if rng.uniform() < 0.5 else -1.0
            m["g1"][I, i, i] = sign * m["omega"][I] * np.sqrt(2.0 * S)
    return m


def model_nn_chain(seed: int = 11, n_modes: int = 3, levels: int = 4) -> dict:
    """Nearest-neighbour chain: the electronic site couples linearly to the
    first mode only; modes couple only to their chain neighbour through a
    bilinear q_I q_{I+1} term that is the identity on the electronic states."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = _empty_model(2, n_modes)
    m["e0"] = np.array([-0.1, 0.1])
    m["v0"] = np.array([[0.0, 0.08], [0.08, 0.0]])
    m["omega"] = rng.uniform(0.08, 0.2, n_modes)
    m["levels"] = np.full(n_modes, levels, dtype=np.int64)
    m["g1"][0, 0, 0] = 0.06
    m["g1"][0, 1, 1] = -0.06
    g2 = []
    for I in range(n_modes - 1):
        v = float(rng.normal(0.0, 0.03))
        for i in range(2):
            g2.append((I, I + 1, i, i, v))
    m["g2"] = g2
    return m


def batch_models(seed: int = 1004, n: int = 64):
    """Coupling scan of uneven 2-state models: mode counts U{8..40}, max bond
    dims U{16..96}, all couplings scaled by s_b, log-spaced over 0.5..2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    scales = np.logspace(np.log10(0.5), np.log10(2.0), n)
    out = []
    for b in range(n):
        n_modes = int(rng.integers(8, 41))
        m_max = int(rng.integers(16, 97))
        m = model_small_2state(seed=seed * 1000 + b, n_modes=n_modes, levels=8)
        m["g1"] = m["g1"] * scales[b]
        m["v0"] = m["v0"] * scales[b]
        out.append((m, m_max))
    return out


def upper_state_index(model: dict) -> int:
    """Index of the initially populated electronic state: the highest-energy
    state for the 2-state models (|S2>), state 0 (LE) otherwise."""
    if model["n_el"] == 2:
        return int(np.argmax(model["e0"]))
    return 0


def product_state_indices(model: dict, el_state: int | None = None) -> list:
    """Basis index per chain site of the product initial state
    |el_state> (x) |0> on every mode."""
    if el_state is None:
        el_state = upper_state_index(model)
    return [el_state if s < 0 else 0 for s in chain_order(model)]


# ---------------------------------------------------------------- tensors
def random_complex(rng: np.random.Generator, shape, scale: float = 1.0) -> np.ndarray:
    """Complex normal entries (real and imaginary parts N(0, scale^2/2))."""
    a = rng.normal(0.0, scale / np.sqrt(2.0), shape)
    b = rng.normal(0.0, scale / np.sqrt(2.0), shape)
    return a + 1j * b


def random_hermitian_env(rng: np.random.Generator, m: int, w: int) -> np.ndarray:
    """Random environment block E[a', w, a] that is Hermitian in (a', a)
    for every w, as environments of a Hermitian MPO are."""
    x = random_complex(rng, (m, w, m))
    return 0.5 * (x + np.conj(np.transpose(x, (2, 1, 0))))


def random_isometry_rows(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """rows x cols matrix with orthonormal rows (rows <= cols), drawn from a
    complex Gaussian and orthonormalised by a library QR."""
    x = random_complex(rng, (cols, rows))
    q, r = np.linalg.qr(x)
    ph = np.diag(r) / np.abs(np.diag(r))
    q = q * ph[None, :]
    return np.conj(q.T)


def bond_caps(dims, m_max: int) -> list:
    """min(m_max, full dimension) of every bond of a chain with site dims."""
    out = []
    n = len(dims)
    for b in range(n - 1):
        left = 1
        for d in dims[: b + 1]:
            left = min(left * int(d), 1 << 40)
        right = 1
        for d in dims[b + 1:]:
            right = min(right * int(d), 1 << 40)
        out.append(int(min(left, right, m_max)))
    return out


def random_right_canonical_mps(seed: int, dims, m_max: int) -> list:
    """Random MPS with every bond at min(m_max, full dimension): sites
    1..n-1 right-orthonormal (complex Gaussian rows orthonormalised by a
    library QR), site 0 a normalised random tensor. Stands in for a
    bond-saturated state of a long propagation."""
    rng = np.random.Generator(np.random.PCG64(seed))
    D = [1] + bond_caps(dims, m_max) + [1]
    ts = []
    for p, d in enumerate(dims):
        if p == 0:
            t = random_complex(rng, (1, d, D[1]))
            t = t / np.linalg.norm(t)
        else:
            t = random_isometry_rows(rng, D[p], d * D[p + 1]).reshape(D[p], d, D[p + 1])
        ts.append(np.ascontiguousarray(t, dtype=np.complex128))
    return ts
