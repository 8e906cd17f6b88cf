"""The C ABI library loads and exports every symbol include/*.h declares, and
the Python binding's struct mirrors match the C layouts (CPU only: no
compute calls)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"LC_API\s+[\w\s\*]*?\b(lc_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_2608_01503_gb300 as lc

    return lc.load()


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("lc_cluster", "lc_cluster_host", "lc_local_move", "lc_contract", "lc_objective",
                 "lc_strerror", "lc_default_opts"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib._name]).decode()
    exported = set(re.findall(r"\sT\s(\w+)$", out, re.M))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    for s in declared_symbols():
        assert hasattr(lib, s)


def test_binding_exports_match_header():
    import paper_2608_01503_gb300 as lc

    assert sorted(lc.EXPORTS) == [s for s in declared_symbols() if s in lc.EXPORTS]
    for s in declared_symbols():
        assert hasattr(lc, s) or s == "lc_default_opts", s


def test_struct_layouts_match_c(tmp_path):
    import paper_2608_01503_gb300 as lc

    prog = tmp_path / "sizes.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "lc.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %d\\n\","
        " sizeof(lc_opts),"
        " sizeof(lc_result), sizeof(lc_event), sizeof(lc_csr), offsetof(lc_opts, stream),"
        " offsetof(lc_result, error_detail), sizeof(lc_server_config), offsetof(lc_server_config, opts),"
        " offsetof(lc_opts, tables), offsetof(lc_result, kernel_bytes), offsetof(lc_result, tables_rebuilt),"
        " offsetof(lc_opts, alloc), offsetof(lc_opts, graphs), offsetof(lc_result, scratch_peak_bytes),"
        " (int)LC_K_COUNT);"
        "return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    vals = list(map(int, subprocess.check_output([str(exe)]).split()))
    assert vals == [ctypes.sizeof(lc._Opts), ctypes.sizeof(lc._Result), ctypes.sizeof(lc._Event),
                    ctypes.sizeof(lc._Csr), lc._Opts.stream.offset, lc._Result.error_detail.offset,
                    ctypes.sizeof(lc._ServerConfig), lc._ServerConfig.opts.offset, lc._Opts.tables.offset,
                    lc._Result.kernel_bytes.offset, lc._Result.tables_rebuilt.offset,
                    lc._Opts.alloc.offset, lc._Opts.graphs.offset, lc._Result.scratch_peak_bytes.offset,
                    len(lc.LC_K_NAMES)]


def test_defaults_and_strerror(lib):
    import paper_2608_01503_gb300 as lc

    o = lc._Opts()
    lib.lc_default_opts(ctypes.byref(o))
    assert o.pass_limit == 6 and (o.eps_num, o.eps_den) == (1, 10)
    assert [(o.phi_num[i], o.phi_den[i]) for i in range(6)] == [(3, 4)] * 4 + [(1, 4)] * 2
    assert o.uncoarsen == 1 and o.validate == 1
    assert lc.lc_strerror(0) == "ok"
    assert "symmetric" in lc.lc_strerror(2)
    assert not o.alloc and not o.dealloc and not o.alloc_ctx  # the library's own pool
    assert lc._c_opts(lc.Options(), None).alloc  # the binding passes PyTorch's allocator
    assert not lc._c_opts(lc.Options(allocator="library"), None).alloc
    cfg = lc.lc_server_default_config()
    assert cfg.slots == 4 and cfg.max_batch == 64 and cfg.hbm_budget == 0
    assert cfg.opts.pass_limit == 6


def test_product_path_does_not_reference_oracle():
    """The CUDA path and its binding never import or load the oracle."""
    pkg = os.path.join(ROOT, "paper_2608_01503_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "lc_oracle" not in text and "liboracle" not in text, f


def test_scratch_estimate_matches_the_driver_sizes(lib):
    """lc_scratch_estimate grows with the graph, counts the kept-table
    buffers and rejects bad sizes (no GPU needed: host arithmetic)."""
    import paper_2608_01503_gb300 as lc

    a = lc.lc_scratch_estimate(1000, 10000)
    b = lc.lc_scratch_estimate(2000, 20000)
    assert 0 < a < b
    # at least the level-0 hash table (16 B per stored edge) and 11 int32 arrays per vertex
    assert a >= 16 * 10000 + 44 * 1000
    assert lc.lc_scratch_estimate(1000, 10000, opts=lc.Options(tables=1)) > a
    assert lc.lc_scratch_estimate(1000, 10000, count=8) > a
    assert lib.lc_scratch_estimate(-1, 0, 1, None) == -1
    assert lib.lc_scratch_estimate(10, 0, 0, None) == -1


def test_release_build_is_not_the_checked_build(lib):
    """lc_debug_enabled is 0 and lc_debug_selftest refuses (LC_ERR_ARG)
    before touching the device in the release build."""
    assert lib.lc_debug_enabled() == 0
    detail = ctypes.c_int64(-1)
    assert lib.lc_debug_selftest(None, ctypes.byref(detail)) == 1
    assert detail.value == 0


def test_checked_build_compiles_and_exports_the_same_symbols():
    """The -DLC_DEBUG=1 build cross-compiles, exports every declared symbol
    and reports itself as checked (host calls only)."""
    from paper_2608_01503_gb300 import _build

    path = _build.build(debug=True)
    assert path.endswith("liblc_debug.so")
    out = subprocess.check_output(["nm", "-D", "--defined-only", path]).decode()
    exported = set(re.findall(r"\sT\s(\w+)$", out, re.M))
    assert not [s for s in declared_symbols() if s not in exported]
    dbg = ctypes.CDLL(path)
    dbg.lc_debug_enabled.restype = ctypes.c_int
    assert dbg.lc_debug_enabled() == 1


def test_option_sets_checked_on_the_host():
    """lc_check_opts (host arithmetic, no device): the defaults and every
    cached tuning are valid; malformed schedules, modes and launch settings
    are refused with LC_ERR_ARG."""
    import json

    import paper_2608_01503_gb300 as lc

    lc.lc_check_opts(None)
    with open(lc.TUNING_CACHE) as f:
        cache = json.load(f)
    assert cache, "no cached tuning"
    for key, tuning in cache.items():
        lc.lc_check_opts(lc.tuned_options(tuning))
        lc.lc_check_opts(lc.tuned_options(tuning, graphs=not tuning["graphs"]))
    for kw in (dict(bins=(8, 16, 32, 128, 256, 512, 1024, 2048, 5000)),  # above bin 8's capacity
               dict(bins=(8, 16, 32, 128, 100)),  # decreasing
               dict(hub_chunk=100), dict(hub_chunk=1 << 20),
               dict(ab_threads=(0, 0, 64)), dict(ab_threads=(32,)), dict(ab_threads=(0, 0, 0, 16)),
               dict(tables=1, bins=(8, 16, 32, 128, 256, 512, 1024, 2048, 2048)),
               dict(pass_limit=17), dict(eps=(0, 10)), dict(phi=[(5, 4)]), dict(symmetry=3)):
        with pytest.raises(lc.LCError) as e:
            lc.lc_check_opts(lc.Options(**kw))
        assert e.value.code == 1, kw
    for kw in (dict(ab_threads=(1, 16, 16, 32, 512)), dict(bins=(8, 8, 8, 128, 128, 512, 512, 2048, 4096)),
               dict(tables=1), dict(graphs=True, hub_chunk=4096)):
        lc.lc_check_opts(lc.Options(**kw))
