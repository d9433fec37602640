"""CPU checks of the band network's checkpoint format (include/pothole.h): a file written here from
the documented layout, with zlib's CRC-32, is accepted by the library's host-side check with the
fields it holds; a damaged CRC, a flipped payload byte, a wrong version, a truncated file, a wrong
magic or a missing file is rejected with PD_ERR_INVALID_ARG.  No GPU is needed."""
import ctypes as C
import os
import struct
import zlib

import numpy as np
import pytest

PD_OK, PD_ERR_INVALID_ARG = 0, 1


@pytest.fixture(scope="module")
def lib():
    from paper_2012_10802_gb300 import build
    L = C.CDLL(build.build())
    L.pd_cnn_checkpoint_info.restype = C.c_int
    L.pd_cnn_checkpoint_info.argtypes = [C.c_char_p, C.POINTER(C.c_int), C.POINTER(C.c_longlong),
                                         C.POINTER(C.c_size_t)]
    L.pd_cnn_num_params.restype = C.c_int
    return L


def _file(n, step, state, version=1, magic=b"PDCNNCK\0", seed=0):
    rng = np.random.default_rng(seed)
    body = magic + struct.pack("<IIQQ", version, n, step, len(state))
    for _ in range(3):          # parameters, first and second Adam moments
        body += rng.normal(size=n).astype("<f4").tobytes()
    body += state
    return body + struct.pack("<I", zlib.crc32(body) & 0xFFFFFFFF)


def _info(lib, path):
    n, step, sb = C.c_int(-1), C.c_longlong(-1), C.c_size_t(0)
    st = lib.pd_cnn_checkpoint_info(os.fsencode(str(path)), C.byref(n), C.byref(step),
                                    C.byref(sb))
    return st, n.value, step.value, sb.value


def test_a_well_formed_file_is_accepted(lib, tmp_path):
    n = lib.pd_cnn_num_params()
    assert n == 19682
    p = tmp_path / "ok.ckpt"
    p.write_bytes(_file(n, 1234, b"generator state \x00\x01\x02"))
    assert _info(lib, p) == (PD_OK, n, 1234, 19)
    p.write_bytes(_file(n, 0, b""))            # no caller state
    assert _info(lib, p) == (PD_OK, n, 0, 0)


@pytest.mark.parametrize("damage", ["crc", "payload", "state", "version", "truncated", "magic",
                                    "long", "missing"])
def test_a_damaged_file_is_rejected(lib, tmp_path, damage):
    n = lib.pd_cnn_num_params()
    good = bytearray(_file(n, 77, b"state bytes"))
    p = tmp_path / "bad.ckpt"
    if damage == "crc":
        good[-1] ^= 0x01
    elif damage == "payload":
        good[32 + 4 * 5000] ^= 0x80                 # one parameter's sign bit
    elif damage == "state":
        good[-5] ^= 0x10
    elif damage == "version":
        good = bytearray(_file(n, 77, b"state bytes", version=2))
    elif damage == "truncated":
        good = good[:-100]
    elif damage == "magic":
        good = bytearray(_file(n, 77, b"state bytes", magic=b"PDCNNCX\0"))
    elif damage == "long":
        good = good + b"\0"
    if damage != "missing":
        p.write_bytes(bytes(good))
    assert _info(lib, p)[0] == PD_ERR_INVALID_ARG
