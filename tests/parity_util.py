"""Element-by-element comparisons shared by the GPU parity tests."""
import numpy as np


def rel(a, b, floor=1e-3):
    """Largest element-by-element relative difference of a from b; entries
    smaller than floor x max|b| are compared against that floor."""
    a, b = np.asarray(a), np.asarray(b)
    den = np.maximum(np.abs(b), floor * max(np.abs(b).max(), 1e-300))
    return (np.abs(a - b) / den).max()


def field_errors(mo, st):
    """Node by node: density and temperature relative to the reference value
    at the node, velocity components relative to the largest speed of the
    reference state."""
    umax = max(np.abs(st["ux"]).max(), np.abs(st["uy"]).max(), 1e-300)
    return {"rho": (np.abs(mo["rho"] - st["rho"]) / np.abs(st["rho"])).max(),
            "ux": np.abs(mo["ux"] - st["ux"]).max() / umax,
            "uy": np.abs(mo["uy"] - st["uy"]).max() / umax,
            "T": (np.abs(mo["T"] - st["T"]) / np.abs(st["T"])).max()}
