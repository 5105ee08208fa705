"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/tsdf.h declares, and its exact integer helpers
(packed key, Section 2.1; multiply-xor hash, Section 3.1) match values worked
out by hand from their definitions. Argument validation that returns before any
CUDA call is exercised too."""
import os
import re

import numpy as np
import pytest

from paper_2608_08287_gb300 import build as tb
from paper_2608_08287_gb300 import tsdf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    tb.build_library()
    return tsdf.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tsdf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tsdf_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(tsdf.EXPORTED)


def test_option_ids_match_the_header():
    text = open(os.path.join(ROOT, "include", "tsdf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    ids = {m.group(1).lower(): int(m.group(2))
           for m in re.finditer(r"\bTSDF_OPT_([A-Z0-9_]+)\s*=\s*(\d+)", text)}
    assert ids == tsdf.OPTIONS


def test_packed_key_by_hand(L):
    b = 1 << 20
    assert tsdf.tsdf_block_key(0, 0, 0) == (b << 42) | (b << 21) | b
    assert tsdf.tsdf_block_key(-b, -b, -b) == 0
    assert tsdf.tsdf_block_key(b - 1, b - 1, b - 1) == (1 << 63) - 1
    assert tsdf.tsdf_block_key(1, -2, 3) == ((b + 1) << 42) | ((b - 2) << 21) | (b + 3)
    # x occupies the top 21 bits, z the bottom 21
    assert tsdf.tsdf_block_key(-b, -b, -b + 5) == 5
    assert tsdf.tsdf_block_key(-b + 1, -b, -b) == 1 << 42
    # a valid key is never the empty key
    assert tsdf.tsdf_block_key(b - 1, b - 1, b - 1) != tsdf.EMPTY_KEY


def test_hash_slot_by_hand(L):
    mask = (1 << 16) - 1
    assert tsdf.tsdf_block_slot(0, 0, 0, 1 << 16) == 0
    assert tsdf.tsdf_block_slot(1, 0, 0, 1 << 16) == 73856093 & mask
    assert tsdf.tsdf_block_slot(0, 1, 0, 1 << 16) == 19349669 & mask
    assert tsdf.tsdf_block_slot(0, 0, 1, 1 << 16) == 83492791 & mask
    # negative coordinates wrap as unsigned 32-bit
    assert tsdf.tsdf_block_slot(-1, 0, 0, 1 << 20) == (2 ** 32 - 73856093) & ((1 << 20) - 1)
    # 2*73856093 = 147712186; 3*19349669 = 58049007; xor, then mask 2^12 - 1
    assert tsdf.tsdf_block_slot(2, 3, 0, 1 << 12) == (147712186 ^ 58049007) & 4095
    assert tsdf.tsdf_block_slot(1, 1, 1, 2) == (73856093 ^ 19349669 ^ 83492791) & 1


def test_volume_bytes_layout(L):
    slots, pool = 1 << 16, 16384
    n = tsdf.tsdf_volume_bytes(slots, pool)
    assert n >= 256 + slots * 16 + pool * 12 + 5 * pool * 512 * 4
    assert n <= 256 + slots * 16 + pool * 12 + 5 * pool * 512 * 4 + 8 * 256
    assert n % 256 == 0
    assert tsdf.tsdf_volume_bytes(1000, 10) == 0      # not a power of two
    assert tsdf.tsdf_volume_bytes(16, 32) == 0        # pool larger than the table
    assert tsdf.tsdf_volume_bytes(16, 0) == 0


def test_invalid_arguments_rejected_before_cuda(L):
    for args in [(0.0, 0.04, 1024, 64), (0.01, 0.005, 1024, 64), (0.01, 0.04, 1000, 64),
                 (0.01, 0.04, 1024, 2048), (0.01, 0.04, 1024, 0), (0.001, 0.04, 1024, 64),
                 (float("nan"), 0.04, 1024, 64)]:
        with pytest.raises(tsdf.TsdfError) as e:
            tsdf.tsdf_volume_create(*args)
        assert e.value.status == "INVALID_ARG"
    with pytest.raises(tsdf.TsdfError):
        tsdf.tsdf_volume_create_in(None, 1 << 20, 0.01, 0.04, 1024, 64)
    with pytest.raises(tsdf.TsdfError):
        tsdf.tsdf_volume_create_in(4096 + 8, 1 << 30, 0.01, 0.04, 1024, 64)  # misaligned
    eye = [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1]
    assert tsdf.tsdf_fuse_frame(None, 4096, 8, 8, (1, 1, 0, 0), eye) == "INVALID_ARG"
    assert tsdf.tsdf_volume_status(None) == "INVALID_ARG"
    assert tsdf.tsdf_volume_reset(None) == "INVALID_ARG"
    tsdf.tsdf_volume_destroy(None)


def test_null_handles_rejected_before_cuda(L):
    """Every entry point that takes a volume or batch refuses a null handle
    with INVALID_ARG before any CUDA call (so this runs without a GPU)."""
    eye = [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1]
    intr = (1, 1, 0, 0)
    for name in tsdf.OPTIONS:
        assert tsdf.tsdf_volume_set_option(None, name, 1) == "INVALID_ARG"
        assert tsdf.tsdf_batch_set_option(None, name, 1) == "INVALID_ARG"
    assert tsdf.tsdf_fuse_frame_async(None, 4096, 8, 8, intr, eye) == "INVALID_ARG"
    assert tsdf.tsdf_fuse_frame_host(None, 4096, 8, 8, intr, eye) == "INVALID_ARG"
    assert tsdf.tsdf_fuse_frame_host_noalloc(None, 4096, 8, 8, intr, eye) == "INVALID_ARG"
    assert tsdf.tsdf_allocate_async(None, 4096, 8, 8, intr, eye) == "INVALID_ARG"
    assert tsdf.tsdf_integrate_async(None, 4096, 8, 8, intr, eye) == "INVALID_ARG"
    assert tsdf.tsdf_volume_copy(None, None) == "INVALID_ARG"
    assert tsdf.tsdf_extract_mesh_async(None, None, None, 0, 4096) == "INVALID_ARG"
    st, t = tsdf.tsdf_autotune_frame(None, 4096, 8, 8, intr, eye)
    assert st == "INVALID_ARG" and t is None
    for fn in (tsdf.tsdf_volume_block_count, tsdf.tsdf_export_blocks,
               tsdf.tsdf_volume_table_stats):
        with pytest.raises(tsdf.TsdfError) as e:
            fn(None)
        assert e.value.status == "INVALID_ARG"
    assert tsdf.tsdf_volume_checkpoint_bytes(None) == 0
    assert tsdf.tsdf_volume_save(None) == ("INVALID_ARG", None)
    assert tsdf.tsdf_volume_load(None, np.zeros(64, np.uint8)) == "INVALID_ARG"
    assert tsdf.tsdf_launch_count() == 0          # nothing was launched


def test_status_strings_and_version(L):
    for code, name in tsdf.STATUS.items():
        want = "TSDF_OK" if code == 0 else f"TSDF_ERR_{name}"
        assert tsdf.tsdf_status_string(code) == want
    assert "sm_103a" in tsdf.tsdf_version()
    assert tsdf.tsdf_launch_count() == 0


STRUCTS = ("tsdf_intrinsics", "tsdf_pose", "tsdf_layout", "tsdf_frame", "tsdf_request",
           "tsdf_completion", "tsdf_table_stats", "tsdf_tuning", "tsdf_extract_timing")


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding mirrors has the size and field offsets the C
    compiler gives it from include/tsdf.h (a C program prints them)."""
    import ctypes
    import subprocess
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "tsdf.h"', 'int main(void) {']
    for name in STRUCTS:
        cls = getattr(tsdf, name)
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True,
                                                         text=True, check=True).stdout.split("\n")
               if line)
    for name in STRUCTS:
        cls = getattr(tsdf, name)
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(cls, field).offset, (name, field)
