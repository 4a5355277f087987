"""The C-ABI library builds, loads, exports every entry point include/gh.h
declares, and rejects bad arguments before touching a GPU (CPU only)."""
import ctypes

import pytest

from paper_2307_16550_gb300 import build, gh


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gh.load()


def test_every_declared_entry_point_is_exported(lib):
    names = gh.header_functions()
    assert len(names) >= 14
    for n in ["gh_create", "gh_destroy", "gh_make_maps", "gh_score_grid", "gh_direct_exact", "gh_detect"]:
        assert n in names
    for n in names:
        assert hasattr(lib, n), n
        assert n in gh._SIGNATURES, f"binding has no signature for {n}"


def test_status_strings(lib):
    assert gh.gh_status_str(gh.GH_OK) == "ok"
    assert gh.gh_status_str(gh.GH_EINVAL) == "invalid argument"
    assert gh.gh_status_str(gh.GH_ECUDA) == "CUDA error"
    assert gh.gh_status_str(12345) == "unknown status"


def test_null_context_is_rejected(lib):
    r = ctypes.byref(gh.GhRadar(24e9, 250e6, 1e-4, 64, 32, 4, 0))
    g = ctypes.byref(gh.GhGrid())
    assert lib.gh_make_maps(None, r, 1, None, None, 0) == gh.GH_EINVAL
    assert lib.gh_score_grid(None, r, None, None, 1, None, 0, g, None, None, None) == gh.GH_EINVAL
    assert lib.gh_direct_exact(None, r, None, None, 1, None, g, None, None, None) == gh.GH_EINVAL
    assert lib.gh_detect(None, 0, r, None, None, 1, None, g, 1, None, None, None) == gh.GH_EINVAL
    assert lib.gh_synth(None, r, None, None, 1, 0, None, None, None, None) == gh.GH_EINVAL
    assert lib.gh_coord_table(None, r, None, None, 1, g, None, None, None, None) == gh.GH_EINVAL
    assert lib.gh_set_timing(None, 1) == gh.GH_EINVAL
    assert lib.gh_reset_stats(None) == gh.GH_EINVAL
    assert lib.gh_launch_count(None) == -1
    assert lib.gh_detect_batch(None, 1, None, None, None, None) == gh.GH_EINVAL
    assert lib.gh_score_points(None, r, None, None, 1, None, 0, None, 0, None) == gh.GH_EINVAL
    assert lib.gh_set_batch_tuning(None, 8, 4) == gh.GH_EINVAL
    assert lib.gh_set_batch_tile(None, 8) == gh.GH_EINVAL
    assert lib.gh_batch_tile(None, None) == gh.GH_EINVAL
    assert lib.gh_batch_row_mode(None, None) == gh.GH_EINVAL
    assert lib.gh_set_batch_row_mode(None, 0) == gh.GH_EINVAL
    assert lib.gh_inject_fault(None, gh.GH_ECUDA, 0) == gh.GH_EINVAL
    lib.gh_destroy(None)
    assert lib.gh_create(None, 0, None) == gh.GH_EINVAL


def test_struct_layouts_match_header(lib):
    assert ctypes.sizeof(gh.GhRadar) == 3 * 8 + 4 * 4
    assert ctypes.sizeof(gh.GhGrid) == 8 * 8 + 4 * 4


def test_struct_sizes_agree_with_the_c_compiler(tmp_path):
    """sizeof of the ABI structs as gcc lays them out from include/gh.h."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "gh.h"\n'
                   'int main(void) { printf("%zu %zu %zu\\n", sizeof(gh_radar), sizeof(gh_grid), '
                   'sizeof(gh_frame)); return 0; }\n')
    exe = tmp_path / "sizes"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out] == [ctypes.sizeof(gh.GhRadar), ctypes.sizeof(gh.GhGrid), ctypes.sizeof(gh.GhFrame)]


def test_loaded_library_was_built_from_these_sources(lib):
    """gh_build_id() of the loaded library equals the hash of the sources in
    the tree (and the id file written beside it)."""
    bid = gh.gh_build_id()
    assert len(bid) == 16 and bid == build.source_hash()
    with open(build.LIB + ".id") as f:
        assert f.read().strip() == bid
