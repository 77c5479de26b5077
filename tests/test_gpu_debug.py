"""The HG_DEBUG build (index checks before every global store of the sub-step kernels, failures recorded in the
grid's error word and reported as HG_ERR_BOUNDS): its self-test must catch an index past the array, and every kernel
family must run clean under it and give the release build's results bit for bit (the checks skip nothing on valid
indices).  The debug library runs in a child process (HG_DEBUG=1 selects it at load time)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1602_05700_gb300 as hg  # noqa: E402
from paper_1602_05700_gb300 import _lib  # noqa: E402
from paper_1602_05700_gb300.builder import LIB_DEBUG, build  # noqa: E402
from tests import debug_cases  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_release_build_has_no_checks():
    assert not hg.is_debug_build()
    g = hg.Grid.unit_cube(16)
    with pytest.raises(hg.HGError) as e:
        g.check_bounds()
    assert e.value.code == _lib.HG_ERR_STATE
    g.free()


@pytest.fixture(scope="module")
def debug_run(tmp_path_factory):
    build(debug=True)
    assert os.path.exists(LIB_DEBUG)
    out = tmp_path_factory.mktemp("debug") / "cases.npz"
    script = ("import sys; sys.path.insert(0, %r)\n"
              "import paper_1602_05700_gb300 as hg\n"
              "assert hg.is_debug_build()\n"
              "g = hg.Grid.unit_cube(20)\n"
              "g.check_bounds()\n"           # the check fires on the index past the array, and is reported
              "g.check_bounds()\n"           # and the error word was cleared after the report
              "g.step(3); g.stats()\n"       # a clean run after it
              "g.free()\n"
              "from tests import debug_cases\n"
              "import numpy as np\n"
              "np.savez(%r, **debug_cases.run_cases())\n") % (ROOT, str(out))
    env = dict(os.environ, HG_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", script], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return dict(np.load(out))


def test_debug_build_matches_release_bit_for_bit(debug_run):
    release = debug_cases.run_cases()
    assert sorted(release) == sorted(debug_run)
    for k in release:
        assert np.array_equal(release[k], debug_run[k]), k
