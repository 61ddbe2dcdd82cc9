"""The C ABI without a GPU: the library loads, exports every declared symbol,
its structs match the header's layout, and argument errors come back as codes
with a message (no compute call is made)."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "anns_amp.h")


@pytest.fixture(scope="module")
def abi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_07156_gb300 import abi as a
    return a


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(anns_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("anns_build_index_from_arrays", "anns_search", "anns_free", "anns_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(abi):
    lib = ctypes.CDLL(abi.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(abi.SYMBOLS) <= set(declared_functions())


def test_struct_layouts(abi):
    assert ctypes.sizeof(abi.anns_build_desc) == 5 * 8 + 5 * 8 + 2 * 4
    assert ctypes.sizeof(abi.anns_precision_policy) == 4 * 4 + 4 * 4 + 4 + 4 + 8 + 8
    assert abi.anns_precision_policy.pair_bits.offset == 40
    assert abi.anns_precision_policy.width_map.offset == 48
    assert ctypes.sizeof(abi.anns_predictor) == 4 * (160 + 32 + 1024 + 32 + 160 + 5 + 5 + 5)
    assert ctypes.sizeof(abi.anns_train_cfg) == 4 + 4 + 4 + 4 + 8 + 4 + 4
    assert ctypes.sizeof(abi.anns_tune_result) == 24 and abi.anns_tune_result.qchunk.offset == 16


def test_argument_errors_without_gpu(abi):
    d = abi.anns_build_desc()
    d.n, d.dim, d.nlist, d.M, d.ksub = 10, 12, 2, 5, 256      # 12 % 5 != 0
    with pytest.raises(abi.AnnsError) as e:
        abi.anns_build_index_from_arrays(d)
    assert e.value.code == -1 and "multiple of M" in str(e.value)
    d.M, d.ksub = 4, 16
    with pytest.raises(abi.AnnsError, match="ksub"):
        abi.anns_build_index_from_arrays(d)
    d.ksub, d.M = 256, 256
    d.dim = 256
    with pytest.raises(abi.AnnsError, match="M must be"):
        abi.anns_build_index_from_arrays(d)
    with pytest.raises(abi.AnnsError, match="null index"):
        abi.anns_search(None, None, 1, 1, None, 1, None, None, None, None)
    assert "null index" in abi.anns_last_error()
    abi.anns_free(None)


def test_binding_constants_match_the_header(abi):
    """The binding's copies of the header's limits are the header's values."""
    text = open(HEADER).read()

    def define(name):
        m = re.search(rf"#define {name} (\S+(?: \S+)*?)\s*(?:/\*|$)", text, flags=re.M)
        return eval(m.group(1), {})

    assert abi.STATIC_SCRATCH_FLOATS == define("ANNS_STATIC_SCRATCH_FLOATS")
    assert (abi.MAX_M, abi.MAX_NPROBE, abi.MAX_K) == (define("ANNS_MAX_M"), define("ANNS_MAX_NPROBE"),
                                                      define("ANNS_MAX_K"))


def test_exact_sum_tap_rejects_bad_sizes(abi):
    with pytest.raises(abi.AnnsError, match="n < 1024"):
        abi.anns_debug_exact_sum(None, 1, 1024, None)
    abi.anns_debug_exact_sum(None, 0, 5, None)   # nothing to do: no launch


def test_load_rejects_bad_files_without_a_gpu(abi, tmp_path):
    """anns_load checks the checksum, magic and shapes before any device call."""
    p = tmp_path / "bad.anns"
    with pytest.raises(abi.AnnsError, match="cannot open"):
        abi.anns_load(str(tmp_path / "missing.anns"))
    p.write_bytes(b"short")
    with pytest.raises(abi.AnnsError, match="too short"):
        abi.anns_load(str(p))
    import struct
    body = b"ANNSAMP1" + struct.pack("<II", 1, 0) + struct.pack("<qqqq", 10, 8, 2, 4) + b"\0" * 64

    def fnv(b):
        h = 0xcbf29ce484222325
        for x in b:
            h = ((h ^ x) * 0x100000001b3) & ((1 << 64) - 1)
        return h

    p.write_bytes(body + struct.pack("<Q", fnv(body) ^ 1))
    with pytest.raises(abi.AnnsError, match="checksum"):
        abi.anns_load(str(p))
    bad = b"NOTANNS!" + body[8:]
    p.write_bytes(bad + struct.pack("<Q", fnv(bad)))
    with pytest.raises(abi.AnnsError, match="magic"):
        abi.anns_load(str(p))
    p.write_bytes(body + struct.pack("<Q", fnv(body)))
    with pytest.raises(abi.AnnsError, match="shorter than its shapes"):
        abi.anns_load(str(p))
