"""The C-ABI library builds, loads and exports every entry point that
include/pcr.h declares (CPU only: no kernel is launched here)."""
import os
import re

import pytest

from conftest import ROOT


def _declared():
    with open(os.path.join(ROOT, "include", "pcr.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^PCR_API\s+[\w\s\*]+?\b(pcr_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_07526_gb300 import build, pcr
    build.build()
    return pcr.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pcr_create", "pcr_destroy", "pcr_set_stream", "pcr_upload_points", "pcr_set_matrix",
                     "pcr_set_viewport", "pcr_set_framebuffer", "pcr_render_basic", "pcr_render_hq",
                     "pcr_resolve", "pcr_reorder_workspace_size", "pcr_reorder_morton_shuffle128",
                     "pcr_status_string", "pcr_last_device_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing


def test_status_strings(lib):
    from paper_2104_07526_gb300 import pcr
    assert pcr.pcr_status_string(0) == "ok"
    assert pcr.pcr_status_string(-3) == "workspace missing or too small"
    assert pcr.pcr_status_string(12345) == "unknown status"


def test_workspace_size_host_only(lib):
    from paper_2104_07526_gb300 import pcr
    sizes = [pcr.pcr_reorder_workspace_size(n) for n in (0, 1, 128, 10_000, 800_000_000)]
    assert sizes == sorted(sizes)
    # points copy (16 B) + two key and two index buffers (4 B each) per point
    assert sizes[-1] >= 800_000_000 * 32
    assert sizes[-1] < 800_000_000 * 34
    with pytest.raises(pcr.PcrError):
        pcr.pcr_reorder_workspace_size(1 << 32)


def test_null_context_is_rejected(lib):
    import ctypes
    assert lib.pcr_render_basic(None, 0, 1) == -1
    assert lib.pcr_set_viewport(None, 4, 4) == -1
    assert lib.pcr_destroy(None) == 0
    out = ctypes.c_uint64()
    assert lib.pcr_reorder_workspace_size(5, None) == -1
    assert lib.pcr_reorder_workspace_size(5, ctypes.byref(out)) == 0


def test_host_only_checks_of_the_later_entry_points(lib):
    """Argument checks that run before any CUDA call: a NULL context or
    output pointer is refused with PCR_ERR_ARG (-1); the batch sizes are
    host computations."""
    import ctypes
    assert lib.pcr_upload_points_mapped(None, None, 0) == -1
    assert lib.pcr_render_rgb(None, 1, 1) == -1
    assert lib.pcr_set_lock_buffer(None, None, 0) == -1
    assert lib.pcr_render_hq1r(None, ctypes.c_float(1.01), 1, 1) == -1
    assert lib.pcr_server_create(None, None, None) == -1
    assert lib.pcr_batch_workspace_size(None) == -1
    assert lib.pcr_batch_num_configs(None) == -1
    size, count = ctypes.c_uint64(), ctypes.c_int()
    assert lib.pcr_batch_workspace_size(ctypes.byref(size)) == 0 and size.value % 256 == 0 and size.value > 0
    assert lib.pcr_batch_num_configs(ctypes.byref(count)) == 0 and count.value >= 1
