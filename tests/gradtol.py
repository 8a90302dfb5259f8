"""Gradient comparison shared by the GPU parity tests (test helper, no GPU).

A gradient entry is a sum of per-pixel terms of both signs, accumulated in
float32 in an order that differs between the two sides (the adjoint adds
with atomics in whatever order the warps reach them; the oracle walks
pixels in raster order).  Where the terms cancel, the entry is small but
its rounding error is that of its largest terms, so a pure relative bar
fails on entries near zero.  grad_close therefore measures

    |a - b| / (|b| + floor * max|b|)

against rtol.  Two floors:

FLOOR (1e-4) -- the adjoint against the oracle on small images (a few
thousand pixels).  With the 1e-3 bar the absolute allowance at a cancelled
entry is 1e-7 of the tensor's largest entry, about one float32 ulp of it
(2^-23 = 1.19e-7).  On a GB300 the worst such comparison reaches 0.30 of
the bar.

WIDE (1e-2) -- full-size images (680 x 1200 and up), where one Gaussian
gathers terms from up to hundreds of thousands of pixels and the rounding
of the cancelled entries grows with that count (the worst reaches 0.77 of
the 1e-3 bar with this floor and 1.55 of it with a floor of 1e-3); and two
GPU adjoints compared at the ten times tighter rtol 1e-4, both with atomic
accumulation orders that change from run to run (1.1 of that bar with a
floor of 1e-4)."""
import numpy as np

FLOOR = 1e-4
WIDE = 1e-2


def grad_err(a, b, floor=FLOOR):
    """Largest |a - b| / (|b| + floor * max|b|) over the tensor."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = np.abs(b).max() + 1e-30
    return float((np.abs(a - b) / (np.abs(b) + floor * scale)).max())


def grad_close(a, b, rtol, name="", floor=FLOOR):
    err = grad_err(a, b, floor)
    assert err <= rtol, (name, err, floor)
