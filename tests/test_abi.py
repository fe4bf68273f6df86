"""CPU checks of the boundary: the library loads, exports every entry point
include/dinr.h declares, the binding declares a prototype for each, and the
product package never reaches into the oracle."""
import glob
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi():
    from paper_2404_19075_b300 import _abi, build
    if not os.path.exists(_abi.LIB_PATH):
        build.build()
    return _abi


def test_library_exports_every_declared_symbol(abi):
    declared = abi.declared_symbols()
    assert len(declared) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", abi.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(declared) <= exported, set(declared) - exported
    # nothing but the ABI is exported
    assert {s for s in exported if not s.startswith("dinr_")} == set()


def test_binding_covers_the_header(abi):
    assert set(abi.declared_symbols()) == set(abi.PROTOTYPES)
    L = abi.lib()
    for name in abi.declared_symbols():
        assert hasattr(L, name)


def test_param_count_host_function(abi):
    from synthetic import workloads as wl
    L = abi.lib()
    for c in (1, 2, 3, 4):
        net = wl.workload(c).net
        assert L.dinr_param_count(net.n_freq, net.hidden_layers, net.width) == net.n_params
    assert L.dinr_param_count(-1, 3, 64) == -1
    for c in (6, 7):
        net = wl.workload(c).net
        assert L.dinr_param_count_din(net.d_in, net.hidden_layers, net.width) == net.n_params


def test_product_never_imports_the_oracle():
    for path in glob.glob(os.path.join(ROOT, "paper_2404_19075_b300", "**", "*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h")):
            with open(path) as f:
                text = f.read()
            assert "import oracle" not in text and "from oracle" not in text, path
