"""The C-ABI library builds, loads and exports every entry point that
include/otgb.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "otgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "return")))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sinkhorn_divergence", "transport_apply", "cluster_grid", "cluster_kmeans", "otgb_softmin",
              "otgb_create", "otgb_destroy", "otgb_default_params", "otgb_last_error", "otgb_plan_free"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2107_02010_gb300 import build

    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params_without_gpu():
    from paper_2107_02010_gb300 import otgb

    p = otgb.default_params()
    assert p.p == 2 and p.scaling == 0.5 and p.trunc_tau == pytest.approx(27.6) and p.max_iters > 0


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2107_02010_gb300 import build, otgb

    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(otgb, "_lib", None)
    with pytest.raises(RuntimeError):
        otgb.load(build_if_missing=False)


def test_softmin_bindings_reject_mismatched_arguments_before_the_call():
    # the kernels trust the sizes they are given: a short output or a column
    # array that does not match would read or write past device buffers, so
    # the binding refuses such calls before any pointer reaches the library
    import torch

    from paper_2107_02010_gb300 import otgb

    q, p = torch.zeros(10, 3), torch.zeros(7, 3)
    w, pot = torch.ones(7), torch.zeros(7)
    bad = [
        dict(p=torch.zeros(7, 4)),                       # coordinates differ
        dict(w=torch.ones(6)),                           # weights of another length
        dict(pot=torch.zeros(8)),                        # potential of another length
        dict(out=torch.empty(9)),                        # output too short
        dict(old=torch.zeros(11)),                       # old of another length
        dict(w=torch.ones(7, dtype=torch.float64)),      # wrong dtype
        dict(out=torch.empty(10, dtype=torch.int32)),    # wrong output dtype
        dict(),                                          # consistent, but on the CPU
    ]
    for kw in bad:
        args = dict(q=q, p=p, w=w, pot=pot, old=None, out=None)
        args.update(kw)
        with pytest.raises(ValueError):
            otgb.softmin_noalloc(args["q"], args["p"], args["w"], args["pot"], 0.1, old=args["old"],
                                 out=args["out"])
        if "out" not in kw:
            with pytest.raises(ValueError):
                otgb.softmin(None, args["q"], args["p"], args["w"], args["pot"], 0.1, old=args["old"])
