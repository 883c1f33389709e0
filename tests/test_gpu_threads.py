"""Host threads calling the library at once, each on its own CUDA stream.

The launchers keep per-kernel, per-device launch facts (shared-memory limit,
SM count, resident CTAs) that are filled on first use; the first calls of a
fresh process race on them.  A child process starts several threads behind
a barrier so that every kernel family (MNS at three top-level sizes, local
search, exhaustive search on both engines, both decoder paths) is first
launched concurrently, then compares each thread's bytes with the same
work repeated serially."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import threading, sys
import numpy as np
import torch
import paper_1501_02894_gb300 as fic
import synth

jobs = [
    ("mns", 32, 4, dict(), 128, 1),
    ("mns", 16, 4, dict(), 96, 2),
    ("mns", 8, 4, dict(), 64, 3),
    ("mns", 32, 4, dict(phase2=False), 160, 4),
    ("local", 16, 4, dict(local_radius=8, local_step=4), 96, 5),
    ("exhaustive", 8, 8, dict(engine=0, dom_step=4), 64, 6),
    ("exhaustive", 8, 8, dict(engine=1, dom_step=4), 64, 7),
    ("nosearch", 32, 8, dict(), 128, 8),
]

def run(job):
    mode, bmax, bmin, kw, N, seed = job
    s = torch.cuda.Stream()
    img = torch.from_numpy(np.ascontiguousarray(synth.gaussian_scene(N, seed))).cuda()
    torch.cuda.synchronize()
    p = fic.params(mode, bmax, bmin, 8.0, **kw)
    with torch.cuda.stream(s):
        st = fic.fic_encode(img, p, stream=s)
        out = [st.to_host(stream=s)]
        for iters in (1, 6):
            out.append(fic.fic_decode(st, iters, stream=s).cpu().numpy())
    s.synchronize()
    return out

def flat(out):
    h = out[0]
    return (h["records"].tobytes(), h["split"].tobytes(), h["tile_offsets"].tobytes(), h["fits"],
            out[1].tobytes(), out[2].tobytes())

fic.lib()
torch.cuda.init()
barrier = threading.Barrier(len(jobs))
got = [None] * len(jobs)
err = []

def worker(i):
    try:
        barrier.wait()
        got[i] = flat(run(jobs[i]))
    except BaseException as e:
        err.append(repr(e))

ts = [threading.Thread(target=worker, args=(i,)) for i in range(len(jobs))]
for t in ts: t.start()
for t in ts: t.join()
if err:
    print("ERR", err); sys.exit(1)
for i, j in enumerate(jobs):
    want = flat(run(j))
    if got[i] != want:
        print("MISMATCH", j); sys.exit(1)
print("OK", len(jobs))
"""


def test_concurrent_first_calls_from_threads():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "OK 8" in r.stdout
