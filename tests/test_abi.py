"""CPU checks of the C ABI: the library loads, exports every entry point that
include/sdc.h declares, and its host-side collocation data agrees with the
oracle's.  No device work is started here."""

import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(sdc_[a-z_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2311_07206_gb300 import build as b
    b.build()
    from paper_2311_07206_gb300 import binding
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2311_07206_gb300 import binding
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
        assert n in binding.SIGNATURES, "binding lacks " + n


def test_default_options(lib):
    from paper_2311_07206_gb300 import default_options
    o = default_options()
    assert o.alpha == 0.1 and o.cg_rtol == 1e-10 and o.reaction_implicit == 1
    assert o.w_frozen == 0 and o.inject_fault == 0 and o.cg_block_size == 1024
    assert o.cg_pipelined == -1 and o.cg_scaled == 1 and o.drop_rule == 0


@pytest.mark.parametrize("M", range(1, 9))
def test_library_collocation_matches_oracle(lib, M):
    from paper_2311_07206_gb300 import radau
    t1, Q1, H1 = radau(M)
    t2, Q2, H2 = oracle.collocation(M)
    np.testing.assert_allclose(t1, t2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(Q1, Q2, rtol=0, atol=4e-15)
    np.testing.assert_allclose(H1, H2, rtol=0, atol=4e-14)


def test_collocation_rejects_bad_M(lib):
    from paper_2311_07206_gb300 import SdcError, radau
    for M in (0, 9):
        with pytest.raises(SdcError):
            radau(M)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2311_07206_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        binding.load()


@pytest.mark.parametrize("bad", ["self_pair", "kind", "area", "Cm", "robin", "range"])
def test_emi_create_rejects_bad_pairs_before_device_work(lib, bad):
    """sdc_create_emi validates the pair data on the host and returns
    SDC_E_INVALID before any device call (so this runs without a GPU)."""
    from paper_2311_07206_gb300 import Context, SdcError
    from workloads.emi import emi_tiny
    wl = emi_tiny("two_cells")
    emi = dict(pair_k=wl.pair_k.copy(), pair_l=wl.pair_l.copy(), pair_area=wl.pair_area.copy(),
               pair_kind=wl.pair_kind.copy(), robin=wl.robin.copy(), Cm=wl.Cm, g_gap=wl.g_gap)
    if bad == "self_pair":
        emi["pair_l"][3] = emi["pair_k"][3]
    elif bad == "kind":
        emi["pair_kind"][0] = 2
    elif bad == "area":
        emi["pair_area"][1] = 0.0
    elif bad == "Cm":
        emi["Cm"] = -1.0
    elif bad == "robin":
        emi["robin"][5] = np.nan
    else:
        emi["pair_k"][2] = wl.n
    with pytest.raises(SdcError) as e:
        Context(3, wl.mesh.xyz, wl.mesh.elems, sigma=np.eye(3), elem_sigma=wl.mesh.elem_sigma,
                ionic=wl.ionic, M=wl.M, emi=emi)
    assert e.value.status == -1 and "EMI" in str(e.value)


def test_energy_stop_rejected_for_batches_and_bad_rho_before_device_work(lib):
    from paper_2311_07206_gb300 import Batch, Context, SdcError, default_options
    from workloads.emi import emi_tiny
    import workloads as W
    wl = emi_tiny("two_cells")
    with pytest.raises(SdcError) as e:
        Context.from_emi(wl, options=default_options(energy_stop=1, sdc_rho=-0.5))
    assert e.value.status == -1
    sq = W.w0_square(n=9, length=2.5)
    with pytest.raises(SdcError) as e:
        Context.from_workload(sq, options=default_options(energy_stop=1, sdc_rho=1.0))
    assert e.value.status == -1
    with pytest.raises(SdcError) as e:
        Batch([sq, sq], options=default_options(energy_stop=1))
    assert e.value.status == -1 and "batch" in str(e.value)


def test_cg_scaled_and_batch_graph_validation_before_device_work(lib):
    from paper_2311_07206_gb300 import Batch, Context, SdcError, default_options
    import workloads as W
    sq = W.w0_square(n=9, length=2.5)
    o = default_options()
    assert o.cg_scaled == 1 and o.batch_graph == 1
    for bad in (-1, 2):
        with pytest.raises(SdcError) as e:
            Context.from_workload(sq, options=default_options(cg_scaled=bad))
        assert e.value.status == -1
        with pytest.raises(SdcError) as e:
            Batch([sq, sq], options=default_options(batch_graph=bad))
        assert e.value.status == -1


def test_drop_rule_validation_before_device_work(lib):
    """drop_rule 1 (the a priori drop tolerance of Sec. 4.1) needs a given
    contraction rho and is per context, not per batch."""
    from paper_2311_07206_gb300 import Batch, Context, SdcError, default_options
    import workloads as W
    sq = W.w0_square(n=9, length=2.5)
    assert default_options().drop_rule == 0
    for opts in (dict(drop_rule=1), dict(drop_rule=2, sdc_rho=0.05), dict(drop_rule=-1)):
        with pytest.raises(SdcError) as e:
            Context.from_workload(sq, options=default_options(**opts))
        assert e.value.status == -1
    with pytest.raises(SdcError) as e:
        Batch([sq, sq], options=default_options(drop_rule=1, sdc_rho=0.05))
    assert e.value.status == -1 and "batch" in str(e.value)


def test_autotune_rejects_bad_arguments_without_a_device(lib):
    """NULL context or batch is rejected before anything else."""
    import ctypes as C
    from paper_2311_07206_gb300 import binding as B
    L = B.load()
    rep = B.sdc_tune_report()
    assert L.sdc_autotune(None, None, None, 0.0, 0.1, 4, 1e-4, 3, C.byref(rep)) == B.SDC_E_INVALID
    assert L.sdc_batch_autotune(None, None, None, 0.0, 0.1, 4, 1e-4, 3, None) == B.SDC_E_INVALID


def test_checked_build_exports_every_declared_symbol(lib):
    """The checked build (SDC_CHECKED=1: index checks in every kernel gather) links
    and exposes the same entry points as the library."""
    import ctypes
    from paper_2311_07206_gb300 import build as b
    chk = ctypes.CDLL(b.build(checked=True))
    for n in _declared():
        assert hasattr(chk, n), n
