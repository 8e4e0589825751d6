"""The bounds-checked build (needs a GPU): libiqa_checked.so compiles a check
of the geometry of every kernel access (unit and tile bounds, tensor-copy
coordinates and alignment, stage capacity, output indices, generator pixel
indices, merge tile indices); a failed check is counted and the access
skipped.  A battery of launches over every kernel family must leave the count
at zero -- the stand-in, on this GPU, for a memory-checking tool -- and the
product library must report the entry point as unsupported."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_battery_has_no_failed_checks():
    from paper_2501_10653_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, IQA_LIBRARY=lib,
               PYTHONPATH=os.pathsep.join([os.path.join(ROOT, "tests"), ROOT,
                                           os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, "-c", "import checked_battery; checked_battery.main()"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked battery: no failed checks" in r.stdout


def test_product_library_has_no_checks():
    from paper_2501_10653_gb300 import build, iqa
    build.build()
    with pytest.raises(iqa.IqaError) as ei:
        iqa.iqa_debug_violations()
    assert ei.value.status == iqa.IQA_ERR_UNSUPPORTED
