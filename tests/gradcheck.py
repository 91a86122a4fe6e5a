"""Gradient comparison used by the GPU parity tests.

The GPU reverse pass returns float32 gradients of double accumulators; the
oracle's reverse mode runs in double on the same frozen decisions.  Two bounds
per parameter family:
  * every entry within ABS_FRAC of the family's largest |gradient| (the
    M-scaled merge terms make scales across entries differ by ~1e5, so a
    purely relative bound would test round-off of entries that cancel);
  * every entry at least BIG of the family's largest |gradient| within REL
    relative error (the entries that dominate a descent step).
"""
import numpy as np

ABS_FRAC = 1e-5
BIG = 0.01
REL = 1e-4


def compare_grads(got, ref, keys=None, abs_frac=ABS_FRAC, rel=REL, big=BIG):
    """Assert both bounds for every family in ``keys`` (default: all of ref);
    return {family: (max |diff| / max |ref|, max relative error over the big
    entries, number of big entries)}."""
    stats = {}
    for k in (ref.keys() if keys is None else keys):
        g = np.asarray(got[k], np.float64).reshape(-1)
        r = np.asarray(ref[k], np.float64).reshape(-1)
        scale = max(float(np.abs(r).max()) if r.size else 0.0, 1e-6)
        d = np.abs(g - r)
        np.testing.assert_allclose(g, r, rtol=0, atol=abs_frac * scale, err_msg=k)
        bigm = np.abs(r) >= big * scale
        relerr = float((d[bigm] / np.abs(r[bigm])).max()) if bigm.any() else 0.0
        assert relerr <= rel, (k, relerr)
        stats[k] = (float(d.max() / scale) if d.size else 0.0, relerr, int(bigm.sum()))
    return stats
