"""The bounds-checked build (libsynth_checked.so, -DSYNTH_CHECKS) on the GPU:
no index of the fused render or of the adjoint leaves its range on any path
(every device status is SYNTH_OK), its outputs equal the release library's
bit for bit (the checks only add tests, never change a value), and its self-test
shows an out-of-range index refused and reported as SYNTH_ERR_BOUNDS once,
the handle rendering unchanged afterwards. The checked library runs in a
child process (SYNTH_CHECKED=1 selects it for a whole process); this process
renders the same cases through the release library."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_matches_release_and_reports_bounds(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_12922_gb300 import build as b
    b.build()
    b.build(checks=True)
    out = str(tmp_path / "checked.npz")
    env = dict(os.environ, SYNTH_CHECKED="1")
    code = f"from tests._checked_cases import child_main; child_main({out!r})"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    got = dict(np.load(out))

    import paper_2104_12922_gb300 as pkg
    from tests._checked_cases import run_cases
    assert pkg.lib().synth_checked_build() == 0
    ref = run_cases(pkg, torch)
    for k, v in ref.items():
        assert np.array_equal(got[k], v), k

    st = got["selftest_status"].tolist()
    # self-test launched; then BOUNDS reported once and cleared; render after: OK
    assert st == [pkg.SYNTH_OK, pkg.SYNTH_ERR_BOUNDS, pkg.SYNTH_OK, pkg.SYNTH_OK], st
    assert bool(got["selftest_render_unchanged"][0])

    # the release library has no such probe
    s = pkg.Synth(seconds=0.1, max_batch=1)
    assert pkg.lib().synth_selftest_bounds(s.handle, None) == pkg.SYNTH_ERR_UNSUPPORTED
    s.close()
