"""The checked build (LSR_CHECKED): device bounds checks on the grid walks, the
hypothesis samples and the matchers' rows that record the first violation and
skip the access instead of trapping.

- It gives the normal build's results bit for bit, with no violation reported,
  on a full registration (FP32 and tensor-core matching), a batch and the
  stage entry points.
- Its reporting path works: the LSR_INJECT_CHECK probe asks the checks about
  one out-of-range index (no access follows) inside a real registration, which
  then returns LSR_E_CHECK naming the site; the next call is clean.

The checked library runs in a child process (LSR_CHECKED=1 selects it in the
binding), so the two builds never share a process.
"""
import json
import os
import subprocess
import sys

import pytest

gpu = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
import paper_1801_01572_gb300 as lsr
from synth import make_pair
out = {"checked": int(lsr.lib().lsr_checked_build())}
fp = make_pair(0, 0, n_p=3000, n_q=3000)
for name, prec in (("fp32", lsr.MATCH_FP32), ("bf16", lsr.MATCH_BF16)):
    with lsr.Context(0, n_hypotheses=300_000, match_precision=prec) as ctx:
        r = ctx.register_pair(fp.P, fp.Q, fp.vpP, fp.vpQ)
        out[name] = [list(r.T.reshape(-1)), r.inliers, r.survivors, r.best_h]
with lsr.Context(0, n_hypotheses=100_000, batch_streams=2) as ctx:
    pairs = [make_pair(0, i, n_p=1500 + 500 * i, n_q=1800) for i in range(3)]
    res = ctx.register_batch([p.P for p in pairs], [p.Q for p in pairs])
    out["batch"] = [[list(r.T.reshape(-1)), r.inliers] for r in res]
    Rt = np.tile(np.eye(3, 4, dtype=np.float32).reshape(1, 12), (5, 1))
    Rt[:, 3] = np.linspace(-0.02, 0.02, 5)
    cnt, sd = ctx.stage_consensus(fp.P, fp.Q, Rt, 0.0375)
    out["consensus"] = [cnt.tolist(), sd.tolist()]
    N, c, _ = ctx.stage_normals(fp.P, fp.vpP, 0.05)
    out["normals"] = float(np.asarray(N, np.float64).sum())
    # the probe: this registration must report the recorded index, the next must not
    if out["checked"]:
        ctx.debug_inject(lsr.INJECT_CHECK, 1)
        try:
            ctx.register_pair(fp.P, fp.Q, fp.vpP, fp.vpQ)
            out["probe"] = "no error"
        except lsr.LsrError as e:
            out["probe"] = [e.code, str(e)]
        r = ctx.register_pair(fp.P, fp.Q, fp.vpP, fp.vpQ)
        out["after_probe"] = r.status
print("RESULT " + json.dumps(out))
"""


def _run(checked: bool) -> dict:
    env = dict(os.environ)
    env["LSR_CHECKED"] = "1" if checked else "0"
    code = "ROOT = " + repr(ROOT) + "\n" + CHILD
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    line = [ln for ln in p.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


@pytest.fixture(scope="module")
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_01572_gb300 import _build
    _build.build()
    _build.build(checked=True)


@gpu
def test_checked_build_matches_normal_build_and_reports_the_probe(built):
    plain = _run(False)
    chk = _run(True)
    assert plain["checked"] == 0 and chk["checked"] == 1
    for k in ("fp32", "bf16", "batch", "consensus", "normals"):
        assert chk[k] == plain[k], k
    code, msg = chk["probe"]
    assert code == -7 and "probe" in msg, chk["probe"]
    assert chk["after_probe"] == 0


def test_checked_library_builds_and_exports_the_abi():
    """Host-only: the checked library compiles for sm_103a, exports the same
    entry points as the header, and says it is the checked build."""
    import ctypes
    import shutil
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_1801_01572_gb300 import _build, lsr as binding
    path = _build.build(checked=True)
    L = ctypes.CDLL(path)
    for name in binding.ABI_FUNCTIONS:
        assert hasattr(L, name), name
    L.lsr_checked_build.restype = ctypes.c_int
    assert L.lsr_checked_build() == 1
