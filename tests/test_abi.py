"""The C-ABI library builds, loads and exports every entry point include/tfs.h declares
(no GPU needed: no compute call is made here)."""
import os
import re

from paper_2510_19047_b300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(tfs_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_builds_for_sm103a():
    path = build.build()
    assert os.path.exists(path)
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_every_declared_symbol_is_exported():
    decl = declared_symbols()
    assert {"tfs_load_tf_data", "tfs_set_noise_weights", "tfs_eval_statistic",
            "tfs_grad_statistic"} <= decl
    exported = set(binding.exported_symbols()) | {
        n for n in decl if hasattr(binding.load_library(), n)}
    missing = decl - exported
    assert not missing, missing


def test_binding_names_follow_the_abi():
    for name in ("load_tf_data", "set_noise_weights", "eval_statistic", "grad_statistic",
                 "select_top", "ascent_step"):
        assert hasattr(binding.TFS, name)
