"""Moduli selection for a requested accuracy.

`load()` reads the trained network parameters shipped with the package
(moduli_mlp.json, written by train_moduli.py) and hands them to the library,
after which emu_zgemm_tol / emu_cgemm_tol pick N with the network and fall
back to the library's a priori rule when the network is not confident.
"""
import json
import os

from . import emu

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "moduli_mlp.json")


def params(path=PATH):
    with open(path) as f:
        return json.load(f)["params"]


def load(path=PATH):
    """Load the trained weights into the library for the current device."""
    p = params(path)
    if len(p) != emu.emu_mlp_param_count():
        raise ValueError("parameter count mismatch")
    return emu.check(emu.emu_mlp_set_weights(p), "emu_mlp_set_weights")


def unload():
    return emu.check(emu.emu_mlp_set_weights(None), "emu_mlp_set_weights")
