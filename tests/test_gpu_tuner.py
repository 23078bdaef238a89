"""The autotuner's choices (column-pass variant, row-block size of the
real-to-complex pass) persist in a JSON file: a first process times the
variants and writes them, a second process reuses them without new trials
(the file is not rewritten), and the choices do not change the results."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, %r)
from paper_1408_6299_gb300 import lib, synth
c = synth.blobs_2d(64, n_t=4)
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
R = lib.Registration(c["n"], c["n_t"], 1, c["beta"], c["reg"], False, lib.REG_MIXED)
mT = dev(c["mT"]); mR = torch.empty(c["n"], dtype=torch.float64, device="cuda")
R.transport(dev(c["v_true"]), mT, mR)
R.set_images(mT, mR)
R.linearize(dev(c["v_true"]))
H = torch.empty(R.coef_shape(), dtype=torch.float64, device="cuda")
R.hessvec(dev(c["vt"]), H)
np.save(sys.argv[1], H.cpu().numpy())
""" % ROOT


def run(tmp_path, tag, env):
    out = str(tmp_path / f"H_{tag}.npy")
    subprocess.run([sys.executable, "-c", SCRIPT, out], check=True, env=env, timeout=600)
    import numpy as np
    return np.load(out)


def test_tuner_choices_persist_and_are_reused(tmp_path):
    cache = tmp_path / "tune_cache.json"
    env = dict(os.environ, REG_TUNE_CACHE=str(cache))
    H1 = run(tmp_path, "first", env)
    assert cache.exists()
    entries = json.loads(cache.read_text())
    assert any("|rows_r2c|" in k for k in entries) and any("|cols|" in k for k in entries), entries
    mtime = os.stat(cache).st_mtime_ns
    text = cache.read_text()
    H2 = run(tmp_path, "second", env)
    assert os.stat(cache).st_mtime_ns == mtime and cache.read_text() == text  # nothing new to record
    assert (H1 == H2).all()
    # a different (forced) choice gives the same result
    forced = {k: (1 - v if "|rows_r2c|" in k else v) for k, v in entries.items()}
    cache.write_text(json.dumps(forced))
    H3 = run(tmp_path, "forced", env)
    assert (H1 == H3).all()
