"""Helpers shared by the GPU tests (comparison with a relative scale)."""
import numpy as np


def rel_close(got, ref, rtol, what=""):
    got, ref = np.asarray(got), np.asarray(ref)
    scale = max(np.abs(ref).max(), 1e-300)
    err = np.abs(got - ref).max() / scale
    assert err <= rtol, f"{what}: max |got-ref| / max|ref| = {err:.3e} > {rtol:.1e}"
    return err
