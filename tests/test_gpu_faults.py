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


def test_autotune_tunes_the_nonrigid_tile_shape_and_uses_it(tmp_path):
    """Nonrigid: the tuner also picks the energy pass's pixels per lane and the register form; the
    next scan runs that shape (its accounting says so) and equals a scan with the shape fixed."""
    spec = synth.spec_c1()
    spec.n_frames = 6
    F = synth.make_series(spec).frames.cuda()
    ctx = B.Context(B.Config(mode="nonrigid"))
    ctx.set_timing(True)
    best = ctx.autotune(F, exec="persistent")
    shape = ctx.tuned_shape(tuple(F.shape), "persistent")
    assert shape["cluster"] == best and shape["unroll"] in (2, 4) and shape["ctas_per_sm"] in (3, 4)
    tuned, _ = ctx.scan(F, exec="persistent")
    t = ctx.last_timing()
    assert (t["cluster"], t["unroll"], t["ctas_per_sm"]) == (shape["cluster"], shape["unroll"], shape["ctas_per_sm"])
    fixed_ctx = B.Context(B.Config(mode="nonrigid", cluster=shape["cluster"], unroll=shape["unroll"],
                                   ctas_per_sm=shape["ctas_per_sm"]))
    fixed, _ = fixed_ctx.scan(F, exec="persistent")
    assert tuned == fixed
    path = str(tmp_path / "tune.jsonl")
    ctx.autotune_save(path)
    ctx2 = B.Context(B.Config(mode="nonrigid"))
    ctx2.autotune_load(path)
    assert ctx2.tuned_shape(tuple(F.shape), "persistent") == shape
    # a line without the energy-pass fields (older files) loads with them unset
    line = open(path).read().splitlines()[0]
    old = line.split(', "unroll"')[0] + "}\n"
    (tmp_path / "old.jsonl").write_text(old)
    ctx3 = B.Context(B.Config(mode="nonrigid"))
    ctx3.autotune_load(str(tmp_path / "old.jsonl"))
    assert ctx3.tuned_shape(tuple(F.shape), "persistent") == dict(cluster=shape["cluster"], unroll=0, ctas_per_sm=0)
    # a field set in the config is not tuned
    ctx4 = B.Context(B.Config(mode="nonrigid", unroll=2))
    ctx4.autotune(F, exec="persistent")
    assert ctx4.tuned_shape(tuple(F.shape), "persistent")["unroll"] == 2
