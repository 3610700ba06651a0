"""The C-ABI library builds, loads and exports every declared symbol; host-side
argument checks work without a GPU (no compute call is made here)."""
import ctypes
import os
import re

import pytest

import paper_1809_07014_gb300 as pkg
from paper_1809_07014_gb300 import build as cuda_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return pkg.load_library()


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(kmer_\w+)\s*\(", text, flags=re.M)
    return names


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} is declared in include/ but not exported"
    assert set(names) == set(pkg._SIGNATURES), "binding and header disagree"


def test_version_and_strerror(lib):
    assert pkg.kmer_version().count(".") == 2
    for code in range(0, -9, -1):
        assert pkg.kmer_strerror(code)
    assert pkg.kmer_strerror(-99) == "unknown error"


def test_default_params(lib):
    p = pkg.kmer_analysis_default_params(31)
    assert (p.k, p.min_count, p.qual_offset, p.qual_threshold) == (31, 2, 33, 20)
    assert (p.ext_mode, p.t_base, p.err_num, p.err_den, p.t_ext, p.variant) == (0, 2, 1, 10, 2, 0)
    assert ctypes.sizeof(pkg.kmer_analysis_params) == 4 * 10 + 8 + 8 + 4 + 4 + 4 + 4 * 3  # no padding: 80 bytes


@pytest.mark.parametrize("field,value", [
    ("k", 0), ("k", 2), ("k", 128), ("k", 129), ("min_count", 0), ("err_den", 0), ("ext_mode", 2),
    ("variant", 7), ("leaf_bits", 23), ("qual_threshold", 256), ("flags", 8), ("l1_bits", 12),
])
def test_invalid_params_rejected_before_device(lib, field, value):
    p = pkg.make_params(31)
    setattr(p, field, value)
    with pytest.raises(pkg.KmerError) as e:
        pkg.kmer_analysis_create(p)
    assert e.value.code == pkg.KMER_ERR_INVALID_ARG


@pytest.mark.parametrize("field,value", [("min_count", 1), ("variant", 1)])
def test_bloom_gate_needs_min_count_two_and_partitions(lib, field, value):
    """The gate drops k-mers seen once, so it is exact only for min_count >= 2,
    and it feeds the partitioned variant's scatter."""
    p = pkg.make_params(31, flags=pkg.KMER_FLAG_BLOOM_GATE)
    setattr(p, field, value)
    with pytest.raises(pkg.KmerError) as e:
        pkg.kmer_analysis_create(p)
    assert e.value.code == pkg.KMER_ERR_INVALID_ARG


def test_reserved_must_be_zero(lib):
    p = pkg.make_params(31)
    p.reserved[2] = 1
    with pytest.raises(pkg.KmerError) as e:
        pkg.kmer_analysis_create(p)
    assert e.value.code == pkg.KMER_ERR_INVALID_ARG


def test_null_arguments(lib):
    assert lib.kmer_analysis_create(None, None, None) == pkg.KMER_ERR_INVALID_ARG
    out = ctypes.c_void_p()
    # null buffers with reads to pack
    assert lib.kmer_readset_create(None, None, None, 5, 33, 20, pkg.KMER_HOST, None,
                                   ctypes.byref(out)) == pkg.KMER_ERR_INVALID_ARG
    assert lib.kmer_readset_create(None, None, None, 0, 33, 20, 7, None,
                                   ctypes.byref(out)) == pkg.KMER_ERR_INVALID_ARG
    assert lib.kmer_readset_create(None, None, None, 0, 300, 20, 0, None,
                                   ctypes.byref(out)) == pkg.KMER_ERR_INVALID_ARG
    assert lib.kmer_analysis_submit(None, None) == pkg.KMER_ERR_INVALID_ARG
    assert lib.kmer_analysis_query(None, None) == pkg.KMER_ERR_INVALID_ARG
    assert lib.kmer_analysis_copy_results(None, None, None, None, None, 0) == pkg.KMER_ERR_INVALID_ARG
    assert lib.kmer_analysis_get_stats(None, None) == pkg.KMER_ERR_INVALID_ARG
    assert lib.kmer_analysis_reset(None) == pkg.KMER_ERR_INVALID_ARG
    assert lib.kmer_analysis_lookup(None, None, 0, None, pkg.KMER_HOST) == pkg.KMER_ERR_INVALID_ARG
    assert lib.kmer_readset_info(None, None, None) == pkg.KMER_ERR_INVALID_ARG
    assert lib.kmer_analysis_destroy(None) == pkg.KMER_OK
    assert lib.kmer_readset_destroy(None) == pkg.KMER_OK
    assert lib.kmer_last_error_message()


def test_no_device_is_an_error_not_a_fallback(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(pkg.KmerError) as e:
        pkg.kmer_analysis_create(pkg.make_params(21))
    assert e.value.code == pkg.KMER_ERR_NO_DEVICE
