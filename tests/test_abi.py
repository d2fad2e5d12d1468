"""The C-ABI library builds, loads without a GPU, exports every symbol that
include/polyrx.h declares, and its structs have the sizes the binding uses."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "polyrx.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(prx_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def P():
    from paper_1409_7498_gb300 import build, polyrx
    build.build()
    return polyrx


def test_exports_every_declared_symbol(P):
    L = C.CDLL(P.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding wraps every one of them under the same name
    wrapped = [n for n in names
               if n not in ("prx_last_error", "prx_status_string", "prx_batch_last_error")]
    assert all(hasattr(P, n) for n in wrapped), [n for n in wrapped if not hasattr(P, n)]


def test_struct_layouts_match_header(P):
    structs = ["prx_system_desc", "prx_reaction_desc", "prx_bond", "prx_rx_trace",
               "prx_observables", "prx_history_record", "prx_stats", "prx_kernel_time",
               "prx_batch_stats"]
    src = "#include <stdio.h>\n#include \"polyrx.h\"\nint main(void){\n" + "".join(
        f'printf("%zu\\n", sizeof({s}));\n' for s in structs) + "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "sz.c")
        exe = os.path.join(d, "sz")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = [int(v) for v in subprocess.check_output([exe]).split()]
    py = [C.sizeof(P.prx_system_desc), C.sizeof(P.prx_reaction_desc), C.sizeof(P.prx_bond),
          C.sizeof(P.prx_rx_trace), C.sizeof(P.prx_observables), P.HISTORY_DTYPE.itemsize,
          C.sizeof(P.prx_stats), C.sizeof(P.prx_kernel_time), C.sizeof(P.prx_batch_stats)]
    assert sizes == py
    assert P.BOND_DTYPE.itemsize == C.sizeof(P.prx_bond)


def test_status_strings_and_estimate(P):
    L = P.lib()
    assert L.prx_status_string(0) == b"ok"
    assert L.prx_status_string(-4) == b"FENE bond overstretched"
    d = P.make_desc(1_048_576, 107.249, adj_cap=4)
    est = P.prx_estimate_bytes(d)
    assert 150e6 < est < 600e6  # roughly 250 B per bead at 1M beads
    # a reaction cutoff beyond the WCA cutoff widens the Verlet lists
    wide = P.make_reaction(2, 1, 1, 4, 0, 1, -1, 1, 0.1, r_react=1.6)
    narrow = P.make_reaction(2, 1, 1, 4, 0, 1, -1, 1, 0.1, r_react=1.1)
    assert P.prx_estimate_bytes(d, narrow) == est < P.prx_estimate_bytes(d, wide)


def test_library_has_no_cpu_fallback_path():
    """The CUDA sources contain kernels for every step and no host compute
    loop over particles other than marshalling."""
    csrc = os.path.join(ROOT, "paper_1409_7498_gb300", "csrc")
    kernels = set()
    for f in os.listdir(csrc):
        if f.endswith(".cu"):
            kernels |= set(re.findall(r"__global__[^;{]*?\b(kb?_\w+)\s*\(", open(os.path.join(csrc, f)).read()))
    for k in ["k_step_nl", "kb_step_nl", "kb_build_nlist", "kb_rx_find", "k_build_nlist", "k_forces64", "k_integrate64", "k_rebin_keys", "k_rebin_permute", "k_rx_find", "k_rx_select_apply",
              "k_rx_compact4", "kb_rx_compact", "k_obs_hist"]:
        assert k in kernels
    binding = open(os.path.join(ROOT, "paper_1409_7498_gb300", "polyrx.py")).read()
    assert "import oracle" not in binding and "from oracle" not in binding
