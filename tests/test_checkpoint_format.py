"""CPU checks of the checkpoint file format (no GPU): files written here by an
independent writer that follows the documented layout -- 56-byte header,
grid edges, 8 state arrays, FNV-1a checksum over 64-bit words -- are accepted
by the library's host-side verifier, and every kind of damage is rejected."""
import os
import struct

import numpy as np
import pytest

MAGIC = b"PPMLRCK1"


def fnv1a_words(data):
    assert len(data) % 8 == 0
    h = 0xcbf29ce484222325
    for (w,) in struct.iter_unpack("<Q", data):
        h ^= w
        h = (h * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def write_checkpoint(path, n, step, time, precision, gamma=5.0 / 3.0, seed=0):
    rng = np.random.default_rng(seed)
    body = struct.pack("<8sIIiiiiqdd", MAGIC, 1, precision, n[0], n[1], n[2], 0, step, time, gamma)
    assert len(body) == 56
    for d in range(3):
        body += np.cumsum(rng.uniform(0.5, 1.5, n[d] + 1)).astype("<f8").tobytes()
    body += rng.standard_normal(8 * n[0] * n[1] * n[2]).astype("<f8").tobytes()
    body += struct.pack("<Q", fnv1a_words(body))
    with open(path, "wb") as f:
        f.write(body)
    return body


@pytest.fixture(scope="module")
def ppm():
    from paper_1607_02214_gb300 import build, ppmlr
    build.build()
    ppmlr.load()
    return ppmlr


def test_valid_file_is_accepted_with_its_fields(ppm, tmp_path):
    p = tmp_path / "a.ck"
    write_checkpoint(p, (5, 3, 4), 1234, 56.75, 1)
    info = ppm.checkpoint_info(p)
    assert info == {"n": [5, 3, 4], "step": 1234, "time": 56.75, "precision": 1}


@pytest.mark.parametrize("damage", ["flip_state", "flip_header", "flip_checksum", "truncate", "trailing",
                                    "magic", "version", "empty"])
def test_damaged_file_is_rejected(ppm, tmp_path, damage):
    p = tmp_path / "b.ck"
    body = bytearray(write_checkpoint(p, (4, 4, 2), 7, 1.5, 0))
    if damage == "flip_state":
        body[56 + 8 * 13 + 100] ^= 0x10
    elif damage == "flip_header":
        body[40] ^= 0x01                  # the simulated time
    elif damage == "flip_checksum":
        body[-1] ^= 0x80
    elif damage == "truncate":
        body = body[:-9]
    elif damage == "trailing":
        body += b"\0" * 8
    elif damage == "magic":
        body[0:8] = b"PPMLRCK2"
    elif damage == "version":
        body[8] = 2
    elif damage == "empty":
        body = bytearray()
    with open(p, "wb") as f:
        f.write(bytes(body))
    with pytest.raises(ppm.PPMLRError):
        ppm.checkpoint_info(p)


def test_missing_file_is_rejected(ppm, tmp_path):
    with pytest.raises(ppm.PPMLRError):
        ppm.checkpoint_info(os.path.join(tmp_path, "does_not_exist.ck"))
