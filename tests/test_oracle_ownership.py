"""Pins for the oracle's model of the data-ownership scheme (section
"Vector Engine Manager": sync, release, discard and the four rules), each
against what the rules fix for a small program whose values are small
integers (so every result is exact and written out here by hand)."""
import numpy as np
import pytest

import oracle
from oracle.ownership import DEVICE, HOST, HOST_WRITE
from workloads import Const, ProgramBuilder

SHAPE = (4, 6)
A = np.arange(24, dtype=np.float64).reshape(SHAPE) - 7.0   # x's first value
B = (np.arange(24, dtype=np.float64) % 5).reshape(SHAPE)   # another host value


def prog():
    b = ProgramBuilder("own")
    x = b.base("float64", SHAPE)
    y = b.base("float64", SHAPE)
    X, Y = b.whole(x), b.whole(y)
    ops = {
        "y=3x+1": [("MULTIPLY", Y, X, Const(3.0)), ("ADD", Y, Y, Const(1.0))],
        "x=x+y": [("ADD", X, X, Y)],
        "x=2x": [("MULTIPLY", X, X, Const(2.0))],
        "x=5": [("COPY", X, Const(5.0))],
        "x[0]=9": [("COPY", b.view(x, 0, (6,), (1,)), Const(9.0))],
        "SYNC x": [("SYNC", X)], "SYNC y": [("SYNC", Y)],
        "DISCARD x": [("DISCARD", X)], "DISCARD y": [("DISCARD", Y)], "FREE y": [("FREE", Y)],
    }
    p = b.build([x, y])
    return p, x, y, ops


def batch(ops, *names):
    from workloads.program import Instr
    out = []
    for nm in names:
        for op, o, *ins in ops[nm]:
            out.append(Instr(op, o, tuple(ins)))
    return out


def model():
    p, x, y, ops = prog()
    m = oracle.OwnershipModel(p)
    m.attach(x, A)
    m.attach(y, np.zeros(SHAPE))
    return m, x, y, ops


def flat(a):
    return np.asarray(a, dtype=np.float64).reshape(-1).tolist()


def test_attach_gives_the_host_ownership():
    m, x, y, ops = model()
    assert m.state(x) == HOST | HOST_WRITE
    assert flat(m.sync(x)) == flat(A)


def test_sync_gives_the_most_recent_copy():
    """Rule 1 / sync: after a batch wrote y, read access yields the batch's
    value, and then both copies are current."""
    m, x, y, ops = model()
    m.submit(batch(ops, "y=3x+1"))
    assert m.state(y) == DEVICE  # the host copy is stale, the host owns nothing
    assert m.state(x) == DEVICE | HOST  # x was read only: both copies current
    assert flat(m.sync(y)) == flat(3 * A + 1)
    assert m.state(y) == DEVICE | HOST


def test_release_then_host_write_reaches_the_next_batch():
    """Rule 1 / release: write access; what the host then writes is what the
    engine reads next (the engine's old copy is not used)."""
    m, x, y, ops = model()
    m.submit(batch(ops, "x=2x"))
    m.release(x)
    assert m.state(x) == HOST | HOST_WRITE
    assert flat(m.sync(x)) == flat(2 * A)  # release synced first
    m.store(x, B)
    m.submit(batch(ops, "y=3x+1"))
    assert flat(m.sync(y)) == flat(3 * B + 1)


def test_discard_declares_the_host_copy_current():
    """Discard: the host copy has been updated, every other copy is invalid:
    the next batch computes from the host's values."""
    m, x, y, ops = model()
    m.submit(batch(ops, "x=2x"))
    m.sync(x)
    m.store(x, B, declared_by_discard=True)
    m.discard(x)
    assert m.state(x) == HOST | HOST_WRITE
    m.submit(batch(ops, "y=3x+1"))
    assert flat(m.sync(y)) == flat(3 * B + 1)


def test_a_batch_revokes_write_access():
    """Rule 2: the engine may write everything a batch names, so the host
    holds write access to none of it afterwards."""
    m, x, y, ops = model()
    m.submit(batch(ops, "y=3x+1"))
    with pytest.raises(oracle.OracleError):
        m.store(x, B)
    m.release(x)
    m.store(x, B)  # with write access again


def test_in_batch_sync_copies_back_at_that_point():
    """Rule 3: a SYNC inside a batch copies the engine's copy to the host
    copy there; a later write in the batch makes the host copy stale again
    without changing it."""
    m, x, y, ops = model()
    m.submit(batch(ops, "x=2x", "SYNC x"))
    assert m.state(x) == DEVICE | HOST
    assert flat(m.host[x]) == flat(2 * A)
    m.submit(batch(ops, "x=2x", "SYNC x", "x=2x"))
    assert m.state(x) == DEVICE
    assert flat(m.host[x]) == flat(4 * A)
    assert flat(m.sync(x)) == flat(8 * A)


def test_in_batch_discard_drops_the_engine_copy():
    """Rule 3: DISCARD deletes the engine's copy. If the host copy is current
    it keeps the value, and the next batch reads it again; otherwise no copy
    holds a value and read access fails."""
    m, x, y, ops = model()
    m.sync(x)
    m.submit(batch(ops, "y=3x+1", "DISCARD x"))
    assert m.state(x) == HOST
    assert flat(m.sync(x)) == flat(A)
    m.submit(batch(ops, "x=x+y"))
    assert flat(m.sync(x)) == flat(A + 3 * A + 1)
    m.submit(batch(ops, "x=2x", "DISCARD x"))
    assert m.state(x) == 0
    with pytest.raises(oracle.OracleError):
        m.sync(x)
    with pytest.raises(oracle.OracleError):  # nor may a batch read it
        m.submit(batch(ops, "y=3x+1"))
    m.submit(batch(ops, "x=5", "y=3x+1"))  # written whole first: defined again
    assert flat(m.sync(y)) == [16.0] * 24


def test_read_after_discard_in_one_batch_is_rejected_and_changes_nothing():
    m, x, y, ops = model()
    m.sync(x)
    with pytest.raises(oracle.OracleError):
        m.submit(batch(ops, "DISCARD x", "y=3x+1"))
    assert m.state(x) == HOST | HOST_WRITE
    assert m.state(y) == HOST | HOST_WRITE


def test_partial_first_write_keeps_the_host_values():
    """Rule 2: a batch whose first use of a base writes only part of it needs
    the rest of the base's current value (from the host copy); one that
    overwrites every element does not."""
    m, x, y, ops = model()
    m.submit(batch(ops, "x[0]=9", "y=3x+1"))
    want = A.copy()
    want[0, :] = 9.0
    assert flat(m.sync(y)) == flat(3 * want + 1)
    m.release(x)
    m.store(x, B)
    m.submit(batch(ops, "x=5", "y=3x+1"))
    assert flat(m.sync(y)) == [16.0] * 24


def test_free_ends_the_mirror():
    m, x, y, ops = model()
    m.submit(batch(ops, "FREE y"))
    with pytest.raises(oracle.OracleError):
        m.state(y)
    assert m.state(x) == HOST | HOST_WRITE  # x was not named by the batch
