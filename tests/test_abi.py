"""The C-ABI library builds for sm_103a, loads, and exports every symbol
that include/treeray.h declares (no compute calls: this runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "treeray.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(tr_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_lists_the_boundary_calls():
    names = declared_symbols()
    for n in ("tr_build_tree", "tr_walk_map", "tr_ray_sweep", "tr_solve"):
        assert n in names


def test_library_builds_and_exports_every_symbol():
    import paper_2105_09644_gb300 as pkg
    from paper_2105_09644_gb300 import binding
    pkg.build()
    L = binding.load()
    for n in declared_symbols():
        assert hasattr(L, n), f"{n} declared in include/treeray.h but not exported"
    assert sorted(binding.EXPORTED) == declared_symbols()


def test_params_default_without_gpu():
    """tr_params_default is pure host code: the paper's defaults."""
    from paper_2105_09644_gb300 import binding
    p = binding.tr_params_default()
    assert p.theta_lim == 0.5 and p.nside == 2 and p.eta_r == 2
    assert p.alpha_B == 2.7e-13 and p.eps_lim == 1e-2 and p.max_iter == 1
    assert p.theta_if == float("inf") and p.theta_src == float("inf")


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2105_09644_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(ImportError):
        binding.load()
