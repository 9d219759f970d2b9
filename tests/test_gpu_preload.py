"""The LD_PRELOAD interposer: an application's cuBLAS GEMM calls run through
the Ozaki-II emulation (bit-exact against the oracle), calls it cannot take
go to cuBLAS, and OZAKI2_EMU_DISABLE turns it off.  Each case runs a child
process (tests/preload_child.py) with the interposer preloaded."""
import json
import os
import subprocess
import sys

import pytest

from paper_2512_08321_gb300 import build as B

pytestmark = pytest.mark.gpu

CHILD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "preload_child.py")


def _run(extra_env):
    if not os.path.exists(B.PRELOAD):
        B.build_preload()
    env = dict(os.environ)
    env.update(extra_env)
    env["LD_PRELOAD"] = B.PRELOAD
    r = subprocess.run([sys.executable, CHILD], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_interposed_calls_are_emulated_bitexact():
    res = _run({"OZAKI2_EMU_VERBOSE": "1"})
    assert res["resolves_to_interposer"]
    for key in ("zgemm_v2", "cgemm_v2", "dgemm_v2", "sgemm_v2", "gemmex_device_scalars"):
        assert res[key] is True, (key, res)
    assert res["legacy_zgemm"] in (True, "absent"), res
    assert res["forwarded_large_k"] is True
    emulated, forwarded = res["emulated"], res["forwarded"]
    assert emulated[:5] == [1, 1, 1, 1, 1], res          # S, D, C, Z, GemmEx
    assert forwarded[1] == 1, res                         # the k > 2^17 DGEMM


def test_moduli_from_environment():
    res = _run({"OZAKI2_EMU_MODULI_Z": "20", "OZAKI2_EMU_MODULI_C": "6", "OZAKI2_EMU_MODULI_D": "12",
                "OZAKI2_EMU_MODULI_S": "5"})
    for key in ("zgemm_v2", "cgemm_v2", "dgemm_v2", "sgemm_v2", "gemmex_device_scalars"):
        assert res[key] is True, (key, res)


def test_disabled_forwards_everything():
    res = _run({"OZAKI2_EMU_DISABLE": "1"})
    assert sum(res["emulated"]) == 0
    # cuBLAS's own results differ from the emulation's in the last bits
    assert res["zgemm_v2"] is False and res["forwarded_large_k"] is True
