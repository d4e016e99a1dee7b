"""The launch autotuner (every choice it makes keeps the results within the parity bars).

Each case runs in a child process, because the tuner reads its environment
(PBS_TUNE, PBS_TUNE_CACHE, PBS_TUNE_FORCE) once per process:
* a solve on a mesh whose Gram, update and tiled nodal steps all have several
  candidates writes its choices to the cache file given; a second process with
  the same cache makes the same choices without timing anything (the file is
  not rewritten) and returns the same eigenvalues bit for bit;
* the Gram's bank-spread staging stride, forced, passes the Gram parity cases."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

# 128 x 128 rod crystal, four Bloch vectors in flight: the finest nodal level is tiled
# (every tile shape fits), the Gram and update kernels have several candidates
CHILD = r"""
import json, sys
import numpy as np
import torch
import __graft_entry__ as ge
ge.build()
import paper_2304_00337_gb300 as pbs
import pbs_inputs as gi
geom = pbs.Geometry(gi.rod_eps(128, 128))
with pbs.Context(0) as ctx:
    lam, res, it = ctx.solve_path(geom, dict(nev=6, block=8, tol=1e-8, kbatch=4), gi.gxmg_path(4))
print(json.dumps(dict(lam=np.asarray(lam).tolist(), res=float(np.max(res)))))
"""


def _child(env_extra, code=CHILD):
    env = dict(os.environ, **env_extra)
    env["PYTHONPATH"] = os.pathsep.join([ROOT, HERE, env.get("PYTHONPATH", "")])
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_choices_cached_and_reused(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cache = tmp_path / "tune.json"
    first = _child({"PBS_TUNE_CACHE": str(cache), "PBS_TUNE": "1"})
    assert first["res"] <= 1e-8
    choices = json.loads(cache.read_text())
    for prefix in ("gram_df", "update_df|", "update|", "node_down|", "node_up|"):
        assert any(k.startswith(prefix) for k in choices), (prefix, sorted(choices))
    assert all(isinstance(v, int) and v >= 0 for v in choices.values())
    stamp = cache.stat().st_mtime_ns
    second = _child({"PBS_TUNE_CACHE": str(cache), "PBS_TUNE": "1"})
    assert cache.stat().st_mtime_ns == stamp  # nothing was tuned again
    assert np.array_equal(np.asarray(first["lam"]), np.asarray(second["lam"]))


@pytest.mark.parametrize("cand", [2, 3])
def test_gram_bank_spread_stride_forced(cand):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # candidates 2 and 3 of the double-float Gram: the padded stride with the default and
    # the doubled number of partial blocks
    env = dict(os.environ, PBS_TUNE_FORCE=f"gram_df={cand}")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                        os.path.join(HERE, "test_gpu_ops.py") + "::test_gram_matches_oracle",
                        os.path.join(HERE, "test_gpu_eigen.py") + "::test_rod64_path_with_extrapolation"],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
