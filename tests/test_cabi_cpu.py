"""CPU-only checks of the C ABI boundary: the library builds for sm_103a,
loads without a GPU, and exports every entry point include/cdgpu.h declares;
the ctypes structures match the header's layout."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cdgpu.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\**\s*(cd_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["cd_csr_upload", "cd_lpa_run", "cd_louvain_local_move", "cd_louvain_aggregate",
                 "cd_modularity", "cd_louvain_run", "cd_graph_free", "cd_status_string"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_2507_06471_gb300 as cd
    path = cd._build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    L = cd.lib()
    for f in declared_functions():
        assert hasattr(L, f)
    assert set(cd.EXPORTED) == set(declared_functions())


def test_status_strings_and_defaults_without_gpu():
    import paper_2507_06471_gb300 as cd
    p = cd.cd_params_default()
    assert (p.max_iter, p.max_levels, p.threshold, p.tie_keep_current, p.singleton_rule,
            p.use_frontier, p.sched_seed) == (100, 64, 0, 1, 1, 1, 0x5EED5EED)
    assert cd.cd_status_string(cd.CD_EBOUNDS).startswith("column id")
    assert cd.cd_status_string(12345) == "unknown status"


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_struct_layouts_match_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    the C compiler gives the header's struct."""
    import paper_2507_06471_gb300 as cd
    structs = [cd.cd_params, cd.cd_round_trace, cd.cd_kernel_profile, cd.cd_request_result]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cdgpu.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    (tmp_path / "layout.c").write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                           str(tmp_path / "layout.c")])
    got = dict(ln.split() for ln in subprocess.check_output([str(exe)], text=True).splitlines())
    for st in structs:
        name = st.__name__
        assert int(got[name]) == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(st, f).offset, (name, f)


def test_oracle_and_generator_build_on_host():
    import oracle
    import synth
    assert os.path.exists(oracle.build())
    # host generator and device generator share one SplitMix64 definition; the
    # host side is checked here, the device side in the GPU tests
    keys = synth.rmat_keys_host(6, 4, "0.57", "0.19", "0.19", seed=3)
    assert keys.shape == (4 << 6,)


def test_upload_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    import paper_2507_06471_gb300 as cd
    off = np.array([0, 1, 2], dtype=np.int64)
    cols = np.array([1, 0], dtype=np.int32)
    with pytest.raises(cd.CDError):
        cd.cd_csr_upload(off, cols, None, stream=0)
