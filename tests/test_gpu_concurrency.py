"""Concurrent solves from several host threads on separate streams (as the
request server runs them) give the same answers as one at a time."""
import threading

import numpy as np
import pytest
import torch

from gpu_util import ctx, dev
from synth import ill_conditioned_problem

pytestmark = pytest.mark.gpu


def test_threads_on_separate_streams_match_serial():
    c = ctx()
    shapes = [(22271, 1024, 4096, 0.0), (60000, 64, 256, 1e-8), (30000, 257, 1028, 0.0), (80000, 128, 512, 1e-10),
              (22271, 512, 2048, 0.0), (40000, 33, 132, 1e-6)]
    probs = []
    for i, (m, n, d, tol) in enumerate(shapes):
        A, b, _ = ill_conditioned_problem(m, n, seed=900 + i, kappa=1e2, noise=1e-3)
        probs.append((dev(A), dev(b), d, tol))
    serial = []
    for A, b, d, tol in probs:
        x, info = c.lstsq(A, b, d, seed=3, tol=tol)
        assert info.status == 0, info.status
        serial.append(x.clone())
    results = [None] * (3 * len(probs))
    errors = []

    def work(k):
        try:
            i = k % len(probs)
            A, b, d, tol = probs[i]
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                x, info = c.lstsq(A, b, d, seed=3, tol=tol, stream=s)
            s.synchronize()
            results[k] = (i, info.status, x)
        except Exception as e:     # surfaced below
            errors.append(repr(e))

    threads = [threading.Thread(target=work, args=(k,)) for k in range(len(results))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for i, status, x in results:
        assert status == 0
        assert torch.equal(x, serial[i])
