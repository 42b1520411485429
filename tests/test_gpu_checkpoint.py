"""Checkpoints: a run saved, resumed in a fresh lattice or batch and continued equals the
uninterrupted run bit for bit, for every storage (needs a GPU)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0911_0459_gb300 import (STORAGE_F16_BLOCKED, STORAGE_F16DEV, STORAGE_F32, STORAGE_F32_BLOCKED,  # noqa: E402
                                   STORAGE_F32_GELIM, STORAGE_F64,
                                   STORAGE_MOMENTS, STORAGE_MOMENTS_F16, Batch, Lattice, LbError)


def capillary(storage):
    return W.Capillary("ck", 200, 37, 64, 120, 5, 27, 12, 8,
                       W.binary_params(nu_l=0.8, nu_g=0.08, storage=storage), theta_deg=50.0)


@pytest.mark.parametrize("storage", [STORAGE_F64, STORAGE_F32, STORAGE_F16DEV, STORAGE_MOMENTS,
                                     STORAGE_MOMENTS_F16, STORAGE_F32_GELIM, STORAGE_F32_BLOCKED,
                                     STORAGE_F16_BLOCKED])
def test_lattice_checkpoint_resumes_bit_for_bit(storage, tmp_path):
    cap = capillary(storage)
    a = Lattice.from_workload(cap)
    a.step(37)                       # odd: the saved state sits in the second buffer
    path = tmp_path / "ck.npz"
    a.save(path)
    a.step(101)                      # graph replays and single launches
    ref, t = a.save_state()
    b = Lattice.from_workload(cap)
    b.load(path)
    assert b.time == 37
    b.step(101)
    got, tb = b.save_state()
    assert tb == t == 138 and np.array_equal(got, ref)
    # a poisoned context takes a checkpoint and runs on
    f, g = b.populations(False) if storage not in (STORAGE_MOMENTS, STORAGE_MOMENTS_F16) else (None, None)
    if f is not None:
        f[0, 10, 70] = np.nan
        b.set_populations(f, g)
        b.step(1)
        with pytest.raises(LbError):
            b.filled_length()
        b.load(path)
        b.step(101)
        assert np.array_equal(b.save_state()[0], ref)
    # checkpoints of another lattice are refused
    with pytest.raises(LbError):
        b.load_state(got[:-1], 0)
    other = Lattice.from_workload(W.Capillary("o", 208, 37, 64, 120, 5, 27, 12, 8,
                                              W.binary_params(storage=storage), theta_deg=50.0))
    with pytest.raises(ValueError):
        other.load(path)
    for x in (a, b, other):
        x.close()


@pytest.mark.parametrize("route", ["load_state", "set_populations", "init_fields"])
def test_a_new_state_clears_a_timed_out_condition(route):
    """A device-side wait that gave up (injected on the host: the context's error word is
    set as the staged kernel sets it) makes the next waiting call return LB_ERR_TIMEOUT and
    refuses steps; each way of giving the lattice a new state clears the word as well as
    the condition, after which reductions and steps work and the run is the saved one."""
    from paper_0911_0459_gb300 import lb as lbmod
    cap = capillary(STORAGE_F32)
    a = Lattice.from_workload(cap)
    a.step(20)
    saved, t = a.save_state()
    f, g = a.populations(False)
    a.step(10)
    ref, _ = a.save_state()
    a.load_state(saved, t)
    a.inject_wait_timeout()
    with pytest.raises(LbError) as e:
        a.filled_length()
    assert e.value.status == lbmod.LB_ERR_TIMEOUT
    with pytest.raises(LbError) as e:
        a.step(1)
    assert e.value.status == lbmod.LB_ERR_STATE
    if route == "load_state":
        a.load_state(saved, t)
    elif route == "set_populations":
        a.set_populations(f, g)
    else:
        a.init_fields(*W.initial_fields(cap))
    a.sync()
    a.filled_length()               # the old timeout is not reported again
    a.filled_length()
    a.step(10)
    if route == "load_state":
        assert np.array_equal(a.save_state()[0], ref)
    assert np.isfinite(a.filled_length()["mass"])
    a.close()


def test_liquid_gas_checkpoint_resumes_bit_for_bit():
    cap = W.config_lg_256x32()
    a = Lattice.from_workload(cap)
    a.step(64)
    buf, t = a.save_state()
    a.step(70)
    b = Lattice.from_workload(cap).load_state(buf, t)
    b.step(70)
    assert np.array_equal(a.save_state()[0], b.save_state()[0])


@pytest.mark.parametrize("storage", [STORAGE_F32, STORAGE_MOMENTS])
def test_batch_checkpoint_resumes_bit_for_bit(storage):
    caps = W.sweep(seed=12, n=4, lengths=(96, 240))
    for c in caps:
        c.nx = c.tube_x0 + c.tube_len
    b1 = Batch(caps, storage=storage)
    b1.step(13)
    buf, t = b1.save_state()
    b1.step(40)
    ref = b1.save_state()[0]
    b2 = Batch(caps, storage=storage)
    b2.load_state(buf, t)
    assert b2.time == 13
    b2.step(40)
    assert b2.time == b1.time and np.array_equal(b2.save_state()[0], ref)
    np.testing.assert_array_equal(b2.lengths(), b1.lengths())
    with pytest.raises(LbError):
        b2.load_state(buf[:-16], 0)
    b1.close()
    b2.close()


def test_runner_resumes_from_its_checkpoint(tmp_path):
    """python -m paper_0911_0459_gb300.run: 300 steps saved and resumed to 500 log the same
    last line as 500 steps in one go."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

    def run(*args):
        r = subprocess.run([sys.executable, "-m", "paper_0911_0459_gb300.run", "--config", "binary_crop_1024x64",
                            "--every", "100", *args], capture_output=True, text=True, cwd=tmp_path, timeout=600,
                           env={**os.environ, "PYTHONPATH": root})
        assert r.returncode == 0, r.stderr[-2000:]
        return [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    first = run("--steps", "300", "--save", "ck.npz")
    assert [x["step"] for x in first] == [100, 200, 300]
    resumed = run("--steps", "500", "--resume", "ck.npz")
    assert [x["step"] for x in resumed] == [400, 500]
    direct = run("--steps", "500")
    for k in ("l", "l_vol", "mass", "phi_sum"):
        assert resumed[-1][k] == direct[-1][k], k
