"""Debugging aids read from the environment (needs a GPU): LR_PLAN forces the plan of searches that
leave it to the library, LR_TIMERS prints each search's stage times.  The library reads the
environment once per process, so each case runs in a child process."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
import datagen, oracle
import paper_2402_13435_b300 as lr
from oracle.compare import check_topk
c = datagen.corpus(71, 40_000, 64, 1024, 12.0, 1.1)
B, K = 20, 30
f = datagen.filters(72, B, c.V, 1.1)
Q = datagen.query_embeddings(72, B, c.d)
po, pid = c.postings()
idx = lr.lr_index_create(torch.from_numpy(c.X).cuda(), c.V, post_off=po, post_ids=pid, n_dense_terms=64,
                         metric="cosine", max_batch=32, max_k=64)
probe = lr.Probe()
ids, sc, cnt = lr.lr_search(idx, torch.from_numpy(Q).cuda(), f, K, probe=probe)
torch.cuda.synchronize()
ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
check_topk(ids.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy(), ref, c.X, Q, c.job_off, c.job_terms, f)
lr.lr_index_destroy(idx)
print(json.dumps({"plan": probe.plan}))
"""


def _run(env_extra):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ)
    env.pop("LR_PLAN", None)
    env.pop("LR_TIMERS", None)
    env.update(env_extra)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    p = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return json.loads(p.stdout.strip().splitlines()[-1]), p.stderr


@pytest.mark.parametrize("forced", ["gemv", "tc"])
def test_lr_plan_forces_the_automatic_plan(forced):
    out, _ = _run({"LR_PLAN": forced})
    assert out["plan"] == forced


def test_lr_timers_prints_stage_times():
    out, err = _run({"LR_TIMERS": "1", "LR_PLAN": "tc"})
    assert out["plan"] == "tc"
    lines = [l for l in err.splitlines() if l.startswith("lr_search B=20 K=30 ms:")]
    assert len(lines) == 1, err[-2000:]
    for stage in ("upload+prep", "sample", "scan", "select", "fallback", "outputs", "total"):
        assert stage in lines[0]


def test_no_timer_lines_without_the_flag():
    out, err = _run({})
    assert not any(l.startswith("lr_search B=") for l in err.splitlines())
