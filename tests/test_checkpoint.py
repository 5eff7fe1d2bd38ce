"""Checkpoint files of load-stepped runs (feti_checkpoint_write / feti_checkpoint_read), host only.

A long load-stepped Newton run (Sec. 5.3 of the paper runs hundreds of load
steps) is resumed from the state (U, step, tau) after its last completed load
step.  These calls touch no GPU, so the format is checked here on the CPU: a
round trip is bit-exact, the header can be read alone, and a truncated,
altered or foreign file is refused with FETI_ERR_IO (13) without touching the
caller's buffer.
"""
import os

import numpy as np
import pytest


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def test_round_trip_is_bit_exact(tmp_path):
    from paper_1508_02599_gb300 import checkpoint_read, checkpoint_write
    rng = np.random.default_rng(3)
    U = rng.normal(size=3 * 1001) * 10.0 ** rng.integers(-300, 300, size=3 * 1001)
    path = tmp_path / "run.ckp"
    checkpoint_write(path, U, 57, 572, 57 / 572)
    V, step, n, tau = checkpoint_read(path)
    assert (step, n, tau) == (57, 572, 57 / 572)
    assert V.tobytes() == U.tobytes()
    assert not os.path.exists(str(path) + ".tmp")
    # overwriting keeps one complete file
    checkpoint_write(path, 2 * U, 58, 572, 58 / 572)
    V, step, _, _ = checkpoint_read(path)
    assert step == 58 and np.array_equal(V, 2 * U)


def test_header_only_and_small_buffer(tmp_path):
    import ctypes as C
    from paper_1508_02599_gb300 import _lib, checkpoint_write
    lib = _lib.load()
    path = tmp_path / "h.ckp"
    checkpoint_write(path, np.arange(30, dtype=float), 3, 10, 0.3)
    info = _lib.FetiCheckpointInfo()
    assert lib.feti_checkpoint_read(str(path).encode(), None, 0, C.byref(info)) == 0
    assert (info.n_dofs, info.step, info.n_load_steps, info.tau) == (30, 3, 10, 0.3)
    buf = np.full(29, -1.0)
    assert lib.feti_checkpoint_read(str(path).encode(), buf.ctypes.data, 29, C.byref(info)) == 1
    assert np.all(buf == -1.0)


@pytest.mark.parametrize("damage", ["truncate", "flip", "magic", "missing"])
def test_damaged_files_are_refused(tmp_path, damage):
    import ctypes as C
    from paper_1508_02599_gb300 import _lib, checkpoint_write
    lib = _lib.load()
    path = tmp_path / "d.ckp"
    U = np.linspace(0.0, 1.0, 300)
    checkpoint_write(path, U, 1, 2, 0.5)
    raw = bytearray(open(path, "rb").read())
    if damage == "truncate":
        raw = raw[:-9]
    elif damage == "flip":
        raw[40 + 8 * 100] ^= 0x01          # one bit of U[100]
    elif damage == "magic":
        raw[0:8] = b"NOTACKP1"
    if damage == "missing":
        os.remove(path)
    else:
        open(path, "wb").write(bytes(raw))
    buf = np.full(300, 7.0)
    st = lib.feti_checkpoint_read(str(path).encode(), buf.ctypes.data, 300, C.byref(_lib.FetiCheckpointInfo()))
    assert st == 13
    assert np.all(buf == 7.0)


def test_invalid_arguments():
    from paper_1508_02599_gb300 import _lib
    lib = _lib.load()
    u = np.zeros(3)
    assert lib.feti_checkpoint_write(None, u.ctypes.data, 3, 0, 1, 0.0) == 1
    assert lib.feti_checkpoint_write(b"/tmp/x.ckp", u.ctypes.data, 3, 5, 4, 1.25) == 1    # step > n_load_steps
    assert lib.feti_checkpoint_write(b"/nonexistent-dir/x.ckp", u.ctypes.data, 3, 1, 4, 0.25) == 13
