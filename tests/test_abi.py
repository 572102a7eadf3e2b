"""CPU-only checks of the C-ABI library: it builds, loads, and exports every entry point include/tdpm.h declares."""
import ctypes
import os
import re

import pytest

from paper_1707_03268_gb300 import build as tbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tdpm.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tdpm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    return tbuild.build()


def test_header_declares_the_pipeline_calls():
    syms = declared_symbols()
    for name in ["tdpm_create", "tdpm_destroy", "tdpm_load_model", "tdpm_decompose", "tdpm_build_pyramid_scores",
                 "tdpm_detect", "tdpm_get_maps", "tdpm_build_batch_scores", "tdpm_get_factors", "tdpm_save_factors", "tdpm_load_factors",
                 "tdpm_release", "tdpm_dt", "tdpm_correlate", "tdpm_last_error"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib_path):
    L = ctypes.CDLL(lib_path)
    missing = [s for s in declared_symbols() if not hasattr(L, s)]
    assert missing == []


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_1707_03268_gb300 import tdpm
    assert sorted(tdpm.SIGNATURES) == declared_symbols()
    tdpm.lib()
    assert "sm_103a" in tdpm.tdpm_version()


def test_struct_layouts_match_header_sizes(lib_path):
    from paper_1707_03268_gb300 import tdpm
    # tdpm_detection: 8 int32/float fields + 2 x 16 int32
    assert ctypes.sizeof(tdpm.Detection) == 4 * (8 + 2 * 16)
    assert ctypes.sizeof(tdpm.Part) == 16 + 8 + 16


def test_create_without_gpu_reports_error(lib_path):
    """With no CUDA device the context cannot be created; the call must return an error, not crash."""
    from paper_1707_03268_gb300 import tdpm
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(tdpm.TdpmError):
        tdpm.tdpm_create(0)


def test_oracle_library_loads():
    from oracle import oracle as orc
    assert orc.num_threads() >= 1


def test_header_struct_sizes_match_the_binding(tmp_path):
    """Compile the header with the host C compiler and compare every public struct's size with its ctypes mirror."""
    import shutil
    import subprocess
    from paper_1707_03268_gb300 import tdpm
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = {"tdpm_detection": tdpm.Detection, "tdpm_level": tdpm.Level, "tdpm_pyramid": tdpm.PyramidDesc,
             "tdpm_part": tdpm.Part, "tdpm_decomp_report": tdpm.DecompReport, "tdpm_request": tdpm.Request,
             "tdpm_server_config": tdpm.ServerConfig, "tdpm_result_info": tdpm.ResultInfo}
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "tdpm.h"\nint main(void){\n' +
                   "".join(f'printf("{n} %zu\\n", sizeof({n}));\n' for n in pairs) + "return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {l.split()[0]: int(l.split()[1]) for l in out if l.strip()}
    for name, cls in pairs.items():
        assert got[name] == ctypes.sizeof(cls), name


@pytest.mark.parametrize("h,w,sbin,lam", [(96, 128, 8, 10), (150, 200, 8, 10), (131, 90, 8, 5), (200, 260, 16, 4)])
def test_hog_pyramid_shape_matches_the_oracle(lib_path, h, w, sbin, lam):
    """The library's HOG pyramid plan (a host computation: level count, sizes, output bytes) against the level
    structure of the oracle's pyramid on an image of the same size."""
    import numpy as np

    from oracle import hog as ohog
    from paper_1707_03268_gb300 import tdpm

    img = np.random.default_rng(h + w).integers(0, 256, size=(h, w, 3)).astype(np.float32)
    want = [tuple(l.shape[:2]) for l in ohog.hog_pyramid(img, sbin=sbin, lam=lam, min_cells=8)]
    shapes, nbytes = tdpm.tdpm_hog_pyramid_shape(h, w, sbin, lam, 8)
    assert shapes == want
    assert nbytes == sum(a * b for a, b in shapes) * 32 * 4


def test_hog_pyramid_shape_rejects_small_images_and_bad_cells(lib_path):
    from paper_1707_03268_gb300 import tdpm

    with pytest.raises(tdpm.TdpmError):
        tdpm.tdpm_hog_pyramid_shape(61, 900, 8, 10, 8)   # no root level has 8 cells on each side
    with pytest.raises(tdpm.TdpmError):
        tdpm.tdpm_hog_pyramid_shape(200, 200, 6, 10, 8)  # cell size not 4, 8 or 16
