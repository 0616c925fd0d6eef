"""The stored oracle registrations (tests/golden/registrations.json) are the
oracle's own results on the generator's pairs: the small entry is recomputed
here and must match bit for bit, every entry's clouds must still be what the
generator makes (digests), and every entry is aligned near the generator's
pose (a sanity bound, not the parity bound: 0.5 deg / 1 cm; config-2
fragments within 1.5 deg / 6 cm, since on small low-overlap fragments the
optimum of the robust objective itself sits centimetres off the generator's
pose -- the 20k + 50k pair 200 by 0.9 deg / 4.9 cm)."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from synth import make_pair, pose_error

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "registrations.json")) as f:
    GOLD = json.load(f)


def test_small_entry_is_the_oracle_result():
    e = GOLD["c0_p0_k0"]
    fp = make_pair(0, 0)
    r = oracle.register(fp.P, fp.Q, fp.vpP, fp.vpQ, diag=True, seed=e["seed"], pair_id=e["pair_id"])
    assert np.array_equal(np.asarray(r["T"]).reshape(-1), np.array(e["T"]))
    for k in ("inliers", "survivors", "n_normal_ok", "best_h", "hyp_inliers", "nn_amb", "hyp_amb", "surv_touch"):
        assert r[k] == e[k], k
    assert r["top"] == e["top"]


@pytest.mark.parametrize("key", sorted(GOLD))
def test_entry_inputs_and_sanity(key):
    e = GOLD[key]
    fp = make_pair(e["config"], e["pair"])
    for X, d in ((fp.P, e["P"]), (fp.Q, e["Q"])):
        assert len(X) == d["n"]
        assert hashlib.sha256(np.ascontiguousarray(X, np.float32).tobytes()).hexdigest()[:16] == d["sha256"]
    assert np.allclose(np.array(e["T_gt"]).reshape(4, 4), fp.T)
    assert e["status"] == 0
    ang, tr = pose_error(np.array(e["T"]).reshape(4, 4), fp.T)
    if e["config"] == 2:
        assert ang < 1.5 and tr < 0.06, (ang, tr)
    else:
        assert ang < 0.5 and tr < 0.01, (ang, tr)
    assert e["hyp_amb"] >= 0 and e["final_amb"] >= 0 and len(e["top"]) == 16
