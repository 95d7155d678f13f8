"""Failure detection without a GPU fault: the persistent executor's bounded wait.

A host-side injection (REG_FAULT_INJECT=stuck_op) leaves one operator waiting
for an input nothing will produce.  The device queue's wait must give up after
REG_QUEUE_TIMEOUT_MS, every worker must leave, reg_scan must report
REG_ETIMEOUT, and the context must stay usable.  Nothing traps, faults or hangs.
"""
import os
import time

import numpy as np
import pytest
import torch

from paper_2010_12478_gb300 import binding as B
from paper_2010_12478_gb300 import synth

pytestmark = pytest.mark.gpu


def test_stuck_operator_times_out_and_context_survives():
    from paper_2010_12478_gb300 import build
    build.build()
    spec = synth.spec_c1()
    spec.n_frames = 8
    F = synth.make_series(spec).frames.cuda()
    ctx = B.Context(B.Config(cluster=2))
    good, _ = ctx.scan(F, exec="persistent")
    os.environ["REG_FAULT_INJECT"] = "stuck_op"
    os.environ["REG_QUEUE_TIMEOUT_MS"] = "300"
    try:
        t0 = time.time()
        with pytest.raises(B.RegError) as e:
            ctx.scan(F, exec="persistent")
        assert e.value.code == B.REG_ETIMEOUT
        assert time.time() - t0 < 10.0
    finally:
        del os.environ["REG_FAULT_INJECT"]
        del os.environ["REG_QUEUE_TIMEOUT_MS"]
    again, _ = ctx.scan(F, exec="persistent")
    assert again == good


def test_autotune_picks_a_valid_size_and_round_trips(tmp_path):
    from paper_2010_12478_gb300 import build
    build.build()
    spec = synth.spec_c1()
    spec.n_frames = 12
    F = synth.make_series(spec).frames.cuda()
    ctx = B.Context(B.Config())
    best = ctx.autotune(F, exec="persistent")
    assert best in (1, 2, 4, 8, 16)
    tuned, _ = ctx.scan(F, exec="persistent")
    fixed, _ = B.Context(B.Config(cluster=best)).scan(F, exec="persistent")
    assert tuned == fixed                      # the tuned size is the one used
    path = str(tmp_path / "tune.jsonl")
    ctx.autotune_save(path)
    ctx2 = B.Context(B.Config())
    ctx2.autotune_load(path)
    assert ctx2.scan(F, exec="persistent")[0] == fixed
