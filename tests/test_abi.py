"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no GPU: no compute calls)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(iqa_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2501_10653_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("iqa_create", "iqa_destroy", "iqa_lisi", "iqa_auglisi", "iqa_both",
                 "iqa_both_host", "iqa_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath],
                         capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = declared_functions() - exported
    assert not missing, "declared but not exported: %s" % sorted(missing)


def test_binding_loads_and_reports_version(libpath):
    from paper_2501_10653_gb300 import iqa
    assert "sm_103a" in iqa.iqa_version()
    p = iqa.iqa_default_params()
    assert (p.C1, p.C2, p.C, p.D) == (1e-6, 1e-6, 1e-6, 0.5e-6)


def test_binding_covers_every_declared_symbol(libpath):
    from paper_2501_10653_gb300 import iqa
    missing = [n for n in declared_functions() if not hasattr(iqa, n)]
    assert not missing, missing


def test_no_gpu_create_fails_loudly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2501_10653_gb300 import iqa
    with pytest.raises(iqa.IqaError) as ei:
        iqa.iqa_create(0, 0)
    assert ei.value.status in (iqa.IQA_ERR_CUDA, iqa.IQA_ERR_INVALID_ARG)


def test_missing_library_raises(tmp_path, monkeypatch):
    from paper_2501_10653_gb300 import iqa
    monkeypatch.setattr(iqa, "_lib", None)
    monkeypatch.setattr(iqa, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        iqa.lib()
