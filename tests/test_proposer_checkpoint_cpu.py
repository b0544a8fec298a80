"""Checkpoint/resume of the proposer's training (host side): the state
written after an epoch reads back unchanged, a checkpoint of another run is
refused, and a write leaves no temporary file behind."""
import os

import numpy as np
import pytest

from paper_2402_16712_gb300 import proposer


def _state(rng):
    P = 97
    return (rng.standard_normal(P).astype(np.float32), rng.standard_normal(P).astype(np.float32),
            np.abs(rng.standard_normal(P)).astype(np.float32))


def test_checkpoint_round_trip(tmp_path):
    rng = np.random.default_rng(3)
    theta, m1, m2 = _state(rng)
    cfg = {"train_seeds": [1, 64], "val_seeds": [30001, 30010], "epochs": 5,
           "batch_instances": 16, "lr": 2e-3, "seed": 0}
    gen = np.random.default_rng(1)
    gen.permutation(10)  # advance: the saved state is mid-stream
    history = [{"epoch": 1, "train_loss": 0.123456789, "val_recall_top32": 0.75}]
    best = (0.75, 1, theta * 2)
    p = str(tmp_path / proposer.CHECKPOINT)
    proposer.save_checkpoint(p, cfg, 1, 4, theta, m1, m2, gen.bit_generator.state, history, best)
    assert os.listdir(tmp_path) == [proposer.CHECKPOINT]  # no temporary file left
    st = proposer.load_checkpoint(p, cfg)
    assert st["epoch"] == 1 and st["step"] == 4 and st["history"] == history
    for a, b in ((st["theta"], theta), (st["m1"], m1), (st["m2"], m2), (st["best"][2], theta * 2)):
        assert a.dtype == np.float32 and np.array_equal(a, b)
    assert st["best"][:2] == (0.75, 1)
    # the permutation stream continues where it stopped
    g2 = np.random.default_rng(99)
    g2.bit_generator.state = st["rng_state"]
    assert np.array_equal(g2.permutation(50), gen.permutation(50))


def test_checkpoint_of_another_run_is_refused(tmp_path):
    rng = np.random.default_rng(4)
    theta, m1, m2 = _state(rng)
    cfg = {"train_seeds": [1, 64], "val_seeds": [30001, 30010], "epochs": 5,
           "batch_instances": 16, "lr": 2e-3, "seed": 0}
    p = str(tmp_path / proposer.CHECKPOINT)
    proposer.save_checkpoint(p, cfg, 2, 8, theta, m1, m2,
                             np.random.default_rng(1).bit_generator.state, [], None)
    st = proposer.load_checkpoint(p, cfg)
    assert st["best"] is None and st["epoch"] == 2
    with pytest.raises(ValueError):
        proposer.load_checkpoint(p, dict(cfg, lr=1e-3))
