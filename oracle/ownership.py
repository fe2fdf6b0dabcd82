"""Reference model of the data-ownership scheme for a base that also has a
copy in host memory (section "Vector Engine Manager": the sync, release
and discard requests and the four rules).

Test infrastructure only (see the package docstring). Plain Python: each
mirrored base has two copies, the engine's (``device``, the oracle's
``Memory``) and the host's (``host``), each either current or not, and the
host either holds write access or not.

* Rule 1: the host asks for access: ``sync`` (read: afterwards the host
  copy is the most recent one), ``release`` (write: the host may change
  its copy; the engine's copy is no longer current), ``discard`` (the host
  has already updated its copy: every other copy is invalid).
* Rule 2: an engine may read every input and write every output its
  instructions name: before a batch, a base whose current value only the
  host copy holds becomes current in the engine (unless the batch's first
  use of it overwrites every element); a base the batch writes has a stale
  host copy afterwards, and the host holds write access to no base the
  batch named.
* Rule 3: an in-batch SYNC copies the engine's copy to the host copy (when
  the engine's copy is current at that point); an in-batch DISCARD deletes
  the engine's copy.
* Rule 4: the model keeps the ownership state (``state``); the host copy
  is read and written only through the calls above.

Readings (where the paper leaves the case open): a batch that reads a
mirrored base after discarding it, while only the host copy holds the
value, is an error (the engine would have to fetch the host copy in the
middle of a batch); a host write without write access is an error; reading
a base no copy holds (by read access or in a batch) is an error.
"""
from __future__ import annotations

import numpy as np

from workloads.program import View

from .interp import CONTROL, Memory, OracleError, execute

DEVICE, HOST, HOST_WRITE = 1, 2, 4


class OwnershipModel:
    """Mirrored bases of one program: ``attach`` gives a base a host copy;
    ``submit`` runs a list of instructions of the program in order."""

    def __init__(self, program):
        self.mem = Memory(program)
        self.host = {}   # base id -> host copy (flat array)
        self.dev = {}    # base id -> engine copy current
        self.hv = {}     # base id -> host copy current
        self.write = {}  # base id -> host holds write access

    # ---------------------------------------------------- the host's side
    def attach(self, bid, values):
        """The host copy holds the base's value; the host owns the base."""
        if bid in self.host:
            raise OracleError("base already has a host copy")
        dt = self.mem.dtype[bid]
        self.host[bid] = np.array(values, dtype=dt).reshape(-1).copy()
        if self.host[bid].size != self.mem.buf[bid].size:
            raise OracleError("host copy size")
        self.dev[bid], self.hv[bid], self.write[bid] = False, True, True

    def sync(self, bid):
        """Read access: returns the host copy, which is current afterwards."""
        self._mirrored(bid)
        if not self.hv[bid]:
            if not self.dev[bid]:
                raise OracleError("no copy holds the base's value")
            self.host[bid] = self.mem.buf[bid].copy()
            self.hv[bid] = True
        return self.host[bid].copy()

    def release(self, bid):
        """Write access: sync, then the engine's copy is not current."""
        self.sync(bid)
        self.dev[bid] = False
        self.write[bid] = True

    def discard(self, bid):
        """The host has updated its copy; every other copy is invalid."""
        self._mirrored(bid)
        self.hv[bid] = True
        self.dev[bid] = False
        self.write[bid] = True

    def store(self, bid, values, declared_by_discard=False):
        """The host writes its copy: allowed with write access, or when a
        ``discard`` declaring the write follows before the next batch."""
        self._mirrored(bid)
        if not (self.write[bid] or declared_by_discard):
            raise OracleError("host write without write access")
        self.host[bid][...] = np.asarray(values, dtype=self.host[bid].dtype).reshape(-1)

    def state(self, bid):
        self._mirrored(bid)
        return (DEVICE if self.dev[bid] else 0) | (HOST if self.hv[bid] else 0) | \
            (HOST_WRITE if self.write[bid] else 0)

    # -------------------------------------------------- the engine's side
    def submit(self, instrs):
        """Execute a batch: rule 2 before and after, rule 3 in between. A
        batch that is rejected changes nothing."""
        # before: which bases take their value from the host copy, checked
        # over the whole batch before anything runs
        dev, hv = dict(self.dev), dict(self.hv)
        fetch, seen = [], set()
        for ins in instrs:
            for bid, kind, covers in self._refs(ins):
                if bid not in self.host:
                    continue
                if bid not in seen:
                    seen.add(bid)
                    needs_old = kind in ("read", "SYNC") or (kind == "write" and not covers)
                    if not dev[bid] and hv[bid] and needs_old:
                        fetch.append(bid)
                        dev[bid] = True
                if kind == "read" and not dev[bid] and hv[bid]:
                    raise OracleError("read of a mirrored base after its discard in the same batch")
                if kind == "read" and not dev[bid]:
                    raise OracleError("read of a mirrored base whose value no copy holds")
                if kind == "write":
                    dev[bid], hv[bid] = True, False
                elif kind == "SYNC" and dev[bid]:
                    hv[bid] = True
                elif kind == "DISCARD":
                    dev[bid] = False
        for bid in fetch:
            self.mem.buf[bid] = self.host[bid].copy()
            self.dev[bid] = True
        for ins in instrs:
            refs = self._refs(ins)
            execute(self.mem, ins)
            for bid, kind, _ in refs:
                if bid not in self.host:
                    continue
                self.write[bid] = False
                if kind == "write":
                    self.dev[bid], self.hv[bid] = True, False
                elif kind == "SYNC" and self.dev[bid]:
                    self.host[bid] = self.mem.buf[bid].copy()
                    self.hv[bid] = True
                elif kind == "DISCARD":
                    self.dev[bid] = False
                elif kind == "FREE":
                    for d in (self.host, self.dev, self.hv, self.write):
                        d.pop(bid, None)

    def value(self, bid):
        """The engine's copy of a base (for bases without a host copy)."""
        return self.mem.buf[bid]

    # ------------------------------------------------------------ helpers
    def _mirrored(self, bid):
        if bid not in self.host:
            raise OracleError("base has no host copy")

    def _refs(self, ins):
        """(base, kind, covers) for every base the instruction names, reads
        first."""
        if ins.op in CONTROL:
            return [(ins.out.base, ins.op, False)]
        out = [(x.base, "read", False) for x in ins.ins if isinstance(x, View)]
        if ins.out is not None:
            n = self.mem.buf[ins.out.base].size if ins.out.base in self.mem.buf else -1
            covers = ins.out.size == n and _one_to_one(ins.out)
            out.append((ins.out.base, "write", covers))
        return out


def _one_to_one(v: View) -> bool:
    """No two indices of the view reach the same element (dimensions sorted
    by |stride|, each stride beyond the span of the smaller ones)."""
    span = 0
    for s, n in sorted((abs(s), n) for n, s in zip(v.shape, v.strides) if n > 1):
        if s <= span:
            return False
        span += s * (n - 1)
    return True


__all__ = ["OwnershipModel", "DEVICE", "HOST", "HOST_WRITE"]
