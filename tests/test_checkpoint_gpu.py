"""Checkpoints on the GPU: a run that saves, and a fresh handle that loads and
continues, give bit for bit the fields, residual and Nusselt number of the
uninterrupted run; files saved with other geometry or parameters, or
corrupted, are refused and leave the handle's state as it was."""

import math

import numpy as np
import pytest

import paper_1908_08386_gb300 as L
from paper_1908_08386_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

MA = 0.1 * math.sqrt(3.0)


def cavity(store, Ra=1e5, mask=True, nx=97, ny=66):
    m = WL.rasterize([("circle", 40.0, 30.0, 16.0)], nx, ny) if mask else None
    return L.Cavity(nx, ny, Ra=Ra, Pr=0.71, Ma=MA, mask=m, store=store)


@pytest.mark.parametrize("store", ["f32", "f16", "f64", "f32x2"])
def test_resume_is_bitwise(tmp_path, store):
    path = tmp_path / "run.ckpt"
    a = cavity(store)
    a.step(301)  # odd: the saved state sits in the second buffer
    a.residual()  # the snapshot the next check compares with
    a.save(path)
    fields_at_save = np.stack(a.fields())
    a.step(259)
    want = np.stack(a.fields()), a.residual(), a.nusselt()

    b = cavity(store)
    b.step(7)  # some other state, to be replaced
    b.load(path)
    assert L.lbmfvm_step_count(b.h) == 301
    assert np.array_equal(np.stack(b.fields()), fields_at_save)
    b.step(259)
    got = np.stack(b.fields()), b.residual(), b.nusselt()
    assert np.array_equal(got[0], want[0])
    assert got[1] == want[1]
    assert got[2][0] == want[2][0] and got[2][2] == want[2][2] and np.array_equal(got[2][1], want[2][1])
    info = L.lbmfvm_checkpoint_info(path)
    assert (info["nx"], info["ny"], info["steps"], info["store"]) == (97, 66, 301, L.PRECISIONS[store])


def test_state_at_step_zero_round_trips(tmp_path):
    path = tmp_path / "rest.ckpt"
    a = cavity("f32")
    a.save(path)
    b = cavity("f32")
    b.step(50)
    b.load(path)
    assert L.lbmfvm_step_count(b.h) == 0
    assert np.array_equal(np.stack(b.fields()), np.stack(a.fields()))
    a.step(100)
    b.step(100)
    assert np.array_equal(np.stack(b.fields()), np.stack(a.fields()))


@pytest.mark.parametrize("other", ["Ra", "mask", "store", "size"])
def test_a_checkpoint_of_another_setup_is_refused(tmp_path, other):
    path = tmp_path / "run.ckpt"
    a = cavity("f32")
    a.step(40)
    a.save(path)
    b = {"Ra": lambda: cavity("f32", Ra=2e5), "mask": lambda: cavity("f32", mask=False),
         "store": lambda: cavity("f16"), "size": lambda: cavity("f32", nx=98)}[other]()
    b.step(3)
    before = np.stack(b.fields())
    with pytest.raises(L.LbmfvmError) as e:
        b.load(path)
    assert e.value.code == L.LBMFVM_ERR_ARG
    assert np.array_equal(np.stack(b.fields()), before)
    assert L.lbmfvm_step_count(b.h) == 3


def test_a_corrupt_checkpoint_is_refused(tmp_path):
    path = tmp_path / "run.ckpt"
    a = cavity("f32")
    a.step(40)
    a.save(path)
    raw = bytearray(path.read_bytes())
    raw[len(raw) // 2] ^= 1
    path.write_bytes(bytes(raw))
    b = cavity("f32")
    b.step(3)
    before = np.stack(b.fields())
    with pytest.raises(L.LbmfvmError) as e:
        b.load(path)
    assert e.value.code == L.LBMFVM_ERR_IO
    assert np.array_equal(np.stack(b.fields()), before)


def test_saving_to_an_unwritable_path_is_an_io_error(tmp_path):
    a = cavity("f32")
    with pytest.raises(L.LbmfvmError) as e:
        a.save(tmp_path / "no_such_dir" / "x.ckpt")
    assert e.value.code == L.LBMFVM_ERR_IO


def test_failed_save_leaves_the_earlier_checkpoint(tmp_path):
    """A save that cannot complete (here: its temporary file cannot be
    created) returns LBMFVM_ERR_IO and leaves the checkpoint already at the
    path loadable and unchanged."""
    path = tmp_path / "keep.ckpt"
    a = cavity("f32")
    a.step(120)
    a.save(path)
    before = path.read_bytes()
    (tmp_path / "keep.ckpt.tmp").mkdir()  # fopen of the temporary file fails
    a.step(80)
    with pytest.raises(L.LbmfvmError) as e:
        a.save(path)
    assert e.value.code == L.LBMFVM_ERR_IO
    assert path.read_bytes() == before
    b = cavity("f32")
    b.load(path)
    assert L.lbmfvm_step_count(b.h) == 120
