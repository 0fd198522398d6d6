"""Checkpoint files without a GPU: the header layout the C header documents,
and lbmfvm_checkpoint_info's verification of magic, sizes and CRC-32s.

The files here are written by the test from the documented layout, with
zlib's crc32 (an implementation independent of the library's) for the
checksums, so a layout or checksum mistake on either side fails."""

import ctypes
import struct
import zlib

import numpy as np
import pytest

import paper_1908_08386_gb300 as L

HEADER_FMT = "<8sII4iq4i4dd6dQII4i76sI"  # the struct's fields in order, no padding


def make_checkpoint(path, nx=7, ny=5, store=L.LBMFVM_F32, steps=1234, seed=0):
    ss = {L.LBMFVM_F64: 8, L.LBMFVM_F32: 4, L.LBMFVM_F16: 2, L.LBMFVM_BF16: 2, L.LBMFVM_F32X2: 8}[store]
    ts = 8 if store in (L.LBMFVM_F64, L.LBMFVM_F32X2) else 4
    n = nx * ny
    payload = np.random.default_rng(seed).integers(0, 256, 2 * 9 * n * ss + n * ts + 2 * n * 8, dtype=np.uint8).tobytes()
    fields = [b"LBMFVMC1", 1, 256, nx, ny, store, 0, steps, 0, 0, 1, 1, 1.0, 0.0, 0.0, 0.0, 0.0,
              0.8, 0.01, 1e-5, 0.5, 0.0, 0.0, len(payload), 0xDEADBEEF, zlib.crc32(payload), 0, 1, 0, 0, bytes(76)]
    head = struct.pack(HEADER_FMT[:-1], *fields)
    head += struct.pack("<I", zlib.crc32(head))
    assert len(head) == 256
    with open(path, "wb") as f:
        f.write(head + payload)
    return head, payload


def test_header_struct_is_256_bytes_with_the_documented_offsets():
    H = L.lbmfvm_checkpoint_header_t
    assert ctypes.sizeof(H) == 256 == struct.calcsize(HEADER_FMT)
    assert H.steps.offset == 32 and H.t_wall.offset == 56 and H.payload_bytes.offset == 144
    assert H.code_crc.offset == 152 and H.payload_crc.offset == 156 and H.header_crc.offset == 252
    assert H.fv_scheme.offset == 160 and H.fv_substeps.offset == 164 and H.energy.offset == 168 and H.wall_bc.offset == 172


@pytest.mark.parametrize("store", [L.LBMFVM_F32, L.LBMFVM_F16, L.LBMFVM_F64, L.LBMFVM_F32X2])
def test_info_reads_a_valid_file(tmp_path, store):
    p = tmp_path / "a.ckpt"
    _, payload = make_checkpoint(p, store=store)
    info = L.lbmfvm_checkpoint_info(p)
    assert (info["nx"], info["ny"], info["store"], info["steps"]) == (7, 5, store, 1234)
    assert info["bc"] == (0, 0, 1, 1) and info["t_wall"] == (1.0, 0.0, 0.0, 0.0)
    assert info["tau"] == 0.8 and info["payload_bytes"] == len(payload)
    assert info["code_crc"] == 0xDEADBEEF and info["payload_crc"] == zlib.crc32(payload)


@pytest.mark.parametrize("where", ["payload", "header", "magic"])
def test_a_flipped_bit_is_an_io_error(tmp_path, where):
    p = tmp_path / "a.ckpt"
    make_checkpoint(p)
    raw = bytearray(p.read_bytes())
    raw[{"payload": 256 + 100, "header": 40, "magic": 0}[where]] ^= 0x10
    p.write_bytes(bytes(raw))
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_checkpoint_info(p)
    assert e.value.code == L.LBMFVM_ERR_IO


@pytest.mark.parametrize("cut", [10, 255, 256, -1])
def test_a_short_file_is_an_io_error(tmp_path, cut):
    p = tmp_path / "a.ckpt"
    make_checkpoint(p)
    raw = p.read_bytes()
    p.write_bytes(raw[:cut] if cut >= 0 else raw[:-1])
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_checkpoint_info(p)
    assert e.value.code == L.LBMFVM_ERR_IO


def test_trailing_bytes_and_a_wrong_payload_size_are_io_errors(tmp_path):
    p = tmp_path / "a.ckpt"
    make_checkpoint(p)
    p.write_bytes(p.read_bytes() + b"\0")
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_checkpoint_info(p)
    assert e.value.code == L.LBMFVM_ERR_IO
    # a header (with a valid CRC) whose payload size disagrees with its grid
    head, payload = make_checkpoint(p)
    bad = bytearray(head[:252])
    struct.pack_into("<Q", bad, 144, len(payload) + 8)
    p.write_bytes(bytes(bad) + struct.pack("<I", zlib.crc32(bytes(bad))) + payload + bytes(8))
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_checkpoint_info(p)
    assert e.value.code == L.LBMFVM_ERR_IO


def test_missing_file_and_null_arguments(tmp_path):
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_checkpoint_info(tmp_path / "none.ckpt")
    assert e.value.code == L.LBMFVM_ERR_IO
    assert L.lib().lbmfvm_checkpoint_info(None, None) == L.LBMFVM_ERR_ARG
    assert L.lib().lbmfvm_save(None, b"x") == L.LBMFVM_ERR_ARG
    assert L.lib().lbmfvm_load(None, b"x") == L.LBMFVM_ERR_ARG
