"""The C-ABI library loads without a GPU and exports every entry point include/chem.h declares;
the generated kernels compile for sm_103a (NVRTC, no GPU needed); host-side argument checks
reject bad input before any launch."""
import os
import re

import pytest

from tests.conftest import ROOT


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "chem.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(chem_[A-Za-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2205_05681_gb300 import chem
    lib = chem.library()
    syms = declared_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(chem.EXPORTS) == syms


def test_spec_errors_are_reported(tmp_path):
    from paper_2205_05681_gb300 import chem
    bad = tmp_path / "bad.mech"
    bad.write_text("ELEMENTS H\nSPECIES 1\nSP H 1.0 1 300 1000 5000 0 0\nREACTIONS 0\nEND\n")
    with pytest.raises(chem.ChemError, match="need at least two species|cannot"):
        chem.compile_only(str(bad))
    with pytest.raises(chem.ChemError, match="cannot open"):
        chem.compile_only(str(tmp_path / "missing.mech"))
    with pytest.raises(chem.ChemError, match="unsupported kernel config"):
        chem.compile_only(os.path.join(ROOT, "tests", "golden", "tiny_hon7.mech"), team=3, block=7)


def test_generated_kernels_compile_for_sm103a(tmp_path):
    from paper_2205_05681_gb300 import chem
    log = chem.compile_only(os.path.join(ROOT, "tests", "golden", "tiny_hon7.mech"), team=32,
                            block=64)
    assert "sm_103a" in log and "chem_integrate_k" in log


@pytest.mark.parametrize("tableau", [1, 2, 3, 4, 5])
def test_every_method_compiles(tmp_path, tableau):
    """ROS3, RODAS3, RODAS4, the explicit RKF45 and the W-method ROS2W generate and compile
    (NVRTC, no GPU)."""
    from paper_2205_05681_gb300 import chem
    log = chem.compile_only(os.path.join(ROOT, "tests", "golden", "tiny_hon7.mech"), team=64,
                            block=64, cache_dir=str(tmp_path), tableau=tableau)
    assert "sm_103a" in log and "chem_integrate_k" in log


def test_adjoint_module_compiles_and_refuses_other_methods(tmp_path):
    from paper_2205_05681_gb300 import chem
    mech = os.path.join(ROOT, "tests", "golden", "tiny_hon7.mech")
    log = chem.compile_only(mech, team=64, block=64, cache_dir=str(tmp_path), adjoint=True)
    assert "chem_adjoint_k" in log and "chem_eval_vjp_k" in log
    with pytest.raises(chem.ChemError, match="adjoint"):
        chem.compile_only(mech, team=64, block=64, cache_dir=str(tmp_path), adjoint=True, tableau=1)
    with pytest.raises(chem.ChemError, match="unknown integration method"):
        chem.compile_only(mech, team=64, block=64, cache_dir=str(tmp_path), tableau=7)


@pytest.mark.parametrize("team,block", [(4, 64), (8, 128), (16, 64)])
def test_subwarp_teams_compile(tmp_path, team, block):
    """Several cells per warp (4-, 8- and 16-lane teams) generate and compile for sm_103a."""
    from paper_2205_05681_gb300 import chem
    log = chem.compile_only(os.path.join(ROOT, "tests", "golden", "tiny_hon7.mech"), team=team,
                            block=block, cache_dir=str(tmp_path))
    assert "sm_103a" in log and "chem_integrate_k" in log
    with pytest.raises(chem.ChemError, match="adjoint"):
        chem.compile_only(os.path.join(ROOT, "tests", "golden", "tiny_hon7.mech"), team=team,
                          block=block, cache_dir=str(tmp_path), adjoint=True)
