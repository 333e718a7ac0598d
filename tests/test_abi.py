"""The C ABI library: builds, loads without a GPU, exports every declared entry point, and validates
arguments before touching the device.  No compute call runs here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lr.h")


@pytest.fixture(scope="module")
def lib_path():
    import importlib.util

    spec = importlib.util.spec_from_file_location("_lr_cuda_build",
                                                  os.path.join(ROOT, "paper_2402_13435_b300", "build.py"))
    build = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(build)  # by path: the package itself loads the library being built
    return build.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(lr_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lr_index_create", "lr_index_destroy", "lr_search", "lr_search_ex", "lr_filter_count",
                 "lr_index_sync", "lr_last_error_message", "lr_version", "lr_index_device_bytes"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    L = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert set(declared_functions()) <= exported


def test_binding_loads_and_reports_version(lib_path):
    import paper_2402_13435_b300 as lr

    assert lr.lr_version() == 201
    assert set(lr.SYMBOLS) <= set(declared_functions())


def test_invalid_arguments_fail_before_any_device_work(lib_path):
    import paper_2402_13435_b300 as lr

    emb = np.zeros((10, 4), dtype=np.float32)
    with pytest.raises(lr.LRError) as e:  # neither bitsets nor postings
        lr.lr_index_create(emb, 8)
    assert e.value.status == lr.LR_ERR_INVALID
    with pytest.raises(lr.LRError) as e:
        lr.lr_index_create(emb, 8, bitsets=np.zeros((10, 1), dtype=np.uint64), max_k=5000)
    assert e.value.status == lr.LR_ERR_INVALID
    with pytest.raises(lr.LRError) as e:
        lr.lr_index_create(np.zeros((10, 300), dtype=np.float32), 8, bitsets=np.zeros((10, 1), dtype=np.uint64))
    assert e.value.status == lr.LR_ERR_UNSUPPORTED
    assert "dim" in lr.lr_last_error_message()
    bits = np.zeros((10, 1), dtype=np.uint64)
    with pytest.raises(lr.LRError) as e:  # precision form: oversample * max_k must fit the selection
        lr.lr_index_create(emb, 8, bitsets=bits, max_k=2000, dtype="fp8", oversample=4)
    assert e.value.status == lr.LR_ERR_INVALID
    assert "oversample" in lr.lr_last_error_message()
    with pytest.raises(lr.LRError) as e:  # the plain form ignores oversample
        lr.lr_index_create(emb, 8, bitsets=bits, max_k=5000, dtype="f32", oversample=4)
    assert "max_k" in lr.lr_last_error_message()


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    import paper_2402_13435_b300 as lr

    monkeypatch.setattr(lr, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError, match="no CPU fallback"):
        lr._load()


def test_key_encoding_host_logic(tmp_path):
    exe = tmp_path / "keys"
    subprocess.check_call(["nvcc", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I",
                           os.path.join(ROOT, "paper_2402_13435_b300", "csrc"),
                           os.path.join(ROOT, "tests", "cpp", "keys_host_test.cu"), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and "OK" in r.stdout, r.stdout


def test_noalloc_rejects_misaligned_and_host_pointers_before_any_device_work(lib_path):
    """lr_search_noalloc checks alignment (pure arithmetic) and then pointer kinds (no GPU here, or on
    a GPU machine plain host addresses): both must fail with LR_ERR_INVALID before any kernel is enqueued."""
    import paper_2402_13435_b300 as lr

    L = lr._lib
    n, d, B, K = 1000, 64, 2, 10
    host = np.zeros((n, d), dtype=np.float32)
    qh = np.zeros((B, d), dtype=np.float32)
    ids = np.zeros((B, K), dtype=np.int32)
    sc = np.zeros((B, K), dtype=np.float32)
    base = host.ctypes.data
    rc = L.lr_search_noalloc(base + 4, n, d, qh.ctypes.data, B, None, 0, K, ids.ctypes.data, sc.ctypes.data, None,
                             None)
    assert rc == lr.LR_ERR_INVALID and "16-byte" in lr.lr_last_error_message()
    rc = L.lr_search_noalloc(base - base % 16, n, d, qh.ctypes.data + 2, B, None, 0, K, ids.ctypes.data,
                             sc.ctypes.data, None, None)
    assert rc == lr.LR_ERR_INVALID and "4-byte" in lr.lr_last_error_message()
    rc = L.lr_search_noalloc(base - base % 16, n, d, qh.ctypes.data, B, None, 0, K, ids.ctypes.data,
                             sc.ctypes.data, None, None)
    assert rc == lr.LR_ERR_INVALID and "device memory" in lr.lr_last_error_message()
    with pytest.raises(ValueError):  # the binding refuses numpy arrays outright
        lr.lr_search_noalloc(host, qh, K, out_ids=ids, out_scores=sc)
