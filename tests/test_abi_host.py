"""Host-side checks of the C ABI: the library loads and exports every entry
point declared in include/vibtdvp.h, and the C++ MPO builder (no GPU needed)
reproduces the Hamiltonian of Sec. 2.2 term by term."""
import os
import re
import subprocess

import numpy as np
import pytest

import vibmodels as vm
from oracle import mpo as ompo
from oracle import vibronic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_1908_10588_gb300 import build
    build.build()
    import paper_1908_10588_gb300 as p
    return p


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "vibtdvp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^(?:vb_status|int|size_t|const char \*)\s*([A-Za-z_][A-Za-z_0-9]*)\s*\(",
                       txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _header_functions()
    for must in ("mpo_build", "mps_create", "tdvp2_sweep", "measure_populations"):
        assert must in names


def test_library_exports_every_declared_symbol(pkg):
    L = pkg.lib()
    names = _header_functions()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    assert set(names) <= exported
    assert set(pkg.EXPORTED) <= exported


def _dense_from_cpp(p, model):
    M = p.Mpo(model)
    W = [M.site_tensor(k) for k in range(M.n_sites)]
    return ompo.mpo_to_dense(W), W


@pytest.mark.parametrize("which", ["c1", "ic", "sf", "nn", "moved"])
def test_cpp_mpo_contracts_to_term_list_hamiltonian(pkg, which):
    models = {
        "c1": vm.model_small_2state(n_modes=3, levels=4),
        "ic": vm.model_internal_conversion(n_modes=4, level_range=(3, 4), n_offdiag=2, n_bilinear=3),
        "sf": vm.model_singlet_fission(n_bath=2, levels=3),
        "nn": vm.model_nn_chain(),
        "moved": dict(vm.model_small_2state(n_modes=3, levels=3), site_order=[1, 0, -1, 2]),
    }
    m = models[which]
    Hd, W = _dense_from_cpp(pkg, m)
    Hs = vibronic.hamiltonian_sparse(m).toarray()
    assert np.max(np.abs(Hd - Hs)) < 1e-13
    assert W[0].shape[0] == 1 and W[-1].shape[3] == 1


def test_cpp_mpo_bond_dims_full_size_models(pkg):
    ic = pkg.Mpo(vm.model_internal_conversion())
    ws = [ic.site_dims(p)[2] for p in range(ic.n_sites - 1)]
    assert max(ws) <= 40 and min(ws) >= 2
    sf = pkg.Mpo(vm.model_singlet_fission())
    assert sf.n_sites == 301
    assert max(sf.site_dims(p)[2] for p in range(300)) <= 12


def test_cpp_mpo_rejects_bad_input(pkg):
    m = vm.model_small_2state(n_modes=2, levels=3)
    with pytest.raises(pkg.VbError):
        pkg.Mpo(dict(m, site_order=[0, 0, -1]))
    bad = dict(m, g2=[(1, 0, 0, 0, 0.1)])
    with pytest.raises(pkg.VbError):
        pkg.Mpo(bad)
    with pytest.raises(pkg.VbError):
        pkg.Mpo(dict(m, levels=np.array([0, 3])))
