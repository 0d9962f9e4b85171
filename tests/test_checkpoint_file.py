"""Checkpoint files checked on the host (alelb_checkpoint_info touches no
device, so this runs without a GPU): a file written by the layout that
include/alelb.h and csrc/checkpoint.cu document is accepted and read back;
truncated, corrupted, extended or foreign files are refused with
ALELB_ERR_ARG and a reason.  The GPU tests write real checkpoints and check
the bitwise resume."""
import struct

import numpy as np
import pytest

from paper_2002_04353_gb300 import alelb

HEAD = struct.Struct("<8sII4iQdq10d6Q")


def _fnv1a(b, h=1469598103934665603):
    for x in b:
        h ^= x
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _write(path, prec=0, N=10, E=4, nstep=7, t=7.0, payload=None):
    ps = 8 if prec == 0 else 4 if prec == 1 else 2
    fs = 8 if prec == 0 else 4
    sec = [18 * N * ps, N * fs, 0 if prec == 0 else 9 * N * 4, 32]
    total = sec[0] + 4 * sec[1] + sec[2] + sec[3]
    if payload is None:
        payload = np.random.default_rng(0).integers(0, 256, total, dtype=np.uint8).tobytes()
    vals = [b"ALELBCK1", 1, 192, prec, 0, N, E, 0x1234, t, nstep,
            1.4, 0.71, 0.02, 1.0, 0.3, 0.1, 0.0, 1000.0, 0.0, 0.0,
            sec[0], sec[1], sec[2], sec[3], total, _fnv1a(payload)]
    head = HEAD.pack(*vals)
    head += struct.pack("<Q", _fnv1a(head))
    assert len(head) == 192
    with open(path, "wb") as fp:
        fp.write(head + payload)
    return head, payload


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_a_well_formed_checkpoint_is_accepted(tmp_path, prec):
    p = tmp_path / "ok.ck"
    _write(p, prec=prec, N=12, E=5, nstep=42, t=41.5)
    info = alelb.checkpoint_info(p)
    assert info == dict(precision=prec, n_nodes=12, n_elems=5, step=42, t=41.5)


def _expect_refused(path, words):
    with pytest.raises(alelb.AlelbError) as e:
        alelb.checkpoint_info(path)
    assert e.value.status == -1  # ALELB_ERR_ARG
    assert words in str(e.value), str(e.value)


def test_truncated_and_corrupted_checkpoints_are_refused(tmp_path):
    p = tmp_path / "ck"
    head, payload = _write(p)
    blob = head + payload
    cases = {
        "ends inside the header": blob[:100],
        "ends inside the payload": blob[:-1],
        "trailing bytes": blob + b"\0",
        "bad magic": b"X" + blob[1:],
        "header checksum": blob[:60] + bytes([blob[60] ^ 1]) + blob[61:],
        "payload checksum": blob[:500] + bytes([blob[500] ^ 0x10]) + blob[501:],
    }
    for words, data in cases.items():
        q = tmp_path / words.replace(" ", "_")
        q.write_bytes(data)
        _expect_refused(q, words)
    _expect_refused(tmp_path / "missing", "cannot open")
    # sizes that do not follow from the header's precision and node count
    q = tmp_path / "sizes"
    h = bytearray(head)
    struct.pack_into("<Q", h, 136, 8)  # pop_bytes
    struct.pack_into("<Q", h, 184, _fnv1a(bytes(h[:184])))
    q.write_bytes(bytes(h) + payload)
    _expect_refused(q, "section sizes")
