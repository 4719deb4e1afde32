"""The C-ABI library builds, loads and exports every entry point that
include/arp.h declares; argument checks that need no GPU."""
import ctypes
import os
import re

import pytest

from _helpers import built_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "arp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(arp_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    path = built_library()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert "arp_create" in syms and "arp_fine_batch" in syms and "arp_parareal_iterate" in syms
    for s in syms:
        assert hasattr(lib, s), s


def test_binding_covers_every_symbol():
    from paper_1303_6615_gb300 import binding
    assert set(declared_symbols()) <= set(binding._SIGS)


def test_query_bytes():
    built_library()
    from paper_1303_6615_gb300 import binding as b
    n1 = b.arp_query_bytes(512, 256, 64, b.ARP_FP64)
    assert n1 > 0
    assert b.arp_query_bytes(512, 512, 64, b.ARP_FP64) > n1
    assert b.arp_query_bytes(500, 256, 64, b.ARP_FP64) == 0
    assert b.arp_query_bytes(4096, 256, 64, b.ARP_FP64) == 0
    assert b.arp_query_bytes(512, 0, 64, b.ARP_FP64) == 0
    assert b.arp_query_bytes(512, 16, 1, b.ARP_FP64) == 0
    assert b.arp_query_bytes(512, 16, 8, 7) == 0


@pytest.mark.parametrize("args,msg", [
    ((500, 1e-2, 1e-4, 4, 0.1, 0.01, 8), "power of two"),
    ((4, 1e-2, 1e-4, 4, 0.1, 0.01, 8), "power of two"),
    ((64, 0.0, 1e-4, 4, 0.1, 0.01, 8), "eps"),
    ((64, 1e-2, -1.0, 4, 0.1, 0.01, 8), "nu"),
    ((64, 1e-2, 1e-4, 0, 0.1, 0.01, 8), "slices"),
    ((64, 1e-2, 1e-4, 4, -0.1, 0.01, 8), "dT"),
    ((64, 1e-2, 1e-4, 4, 0.1, 0.2, 8), "dt"),
    ((64, 1e-2, 1e-4, 4, 0.1, 0.01, 1), "M"),
])
def test_create_rejects_invalid_sizes_without_touching_the_gpu(args, msg):
    built_library()
    from paper_1303_6615_gb300 import binding as b
    with pytest.raises(b.ArpError) as ei:
        b.arp_create(*args)
    assert ei.value.status == b.ARP_EINVAL
    assert msg in str(ei.value)


def test_null_context_is_rejected():
    built_library()
    from paper_1303_6615_gb300 import binding as b
    lib = b.load_library()
    assert lib.arp_fine_batch(None, None, None, 1, None) == b.ARP_EINVAL
    assert lib.arp_set_option(None, 1, 1.0) == b.ARP_EINVAL
    assert lib.arp_destroy(None) == b.ARP_OK
    assert isinstance(lib.arp_last_error(None), bytes)
