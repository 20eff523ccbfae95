"""Shared helpers of the tests (no method arithmetic).

Error measure of a DG state against the oracle: for each variable, the largest
difference of the two cell polynomials anywhere inside a cell,
    max_cells ( |d avg| + sum_d |d (dU/dx_d)| h_d / 2 ),
relative to the variable's scale, max_cells |avg| (for momentum and magnetic
field: the largest vector magnitude of the averages).  Normalising each
coefficient class by its own maximum is ill-posed when a class is identically
zero at the start (the density slopes of the Orszag-Tang vortex are zero, so after
one step they hold only O(dt) values and rounding).
"""
import numpy as np


def _vars(eq, dim):
    """(name, Taylor plane list or magnetic marker) of every variable."""
    nT = 4 if dim == 2 else 5
    names = ["rho", "mx", "my", "E"] if dim == 2 else ["rho", "mx", "my", "mz", "E"]
    return nT, names


def poly_rel_err(got, ref, eq, dim, h):
    """Largest relative polynomial error over the variables; returns (err, name)."""
    nT, names = _vars(eq, dim)
    K = dim + 1
    avg = lambda a, v: a[v * K]
    # scales
    mom = [v for v in range(nT) if names[v].startswith("m")]
    mscale = np.sqrt(sum(avg(ref, v) ** 2 for v in mom)).max()
    worst, where = 0.0, None
    for v in range(nT):
        d = np.abs(avg(got, v) - avg(ref, v))
        for k in range(1, K):
            d = d + np.abs(got[v * K + k] - ref[v * K + k]) * (0.5 * h[k - 1])
        s = mscale if v in mom else np.abs(avg(ref, v)).max()
        e = d.max() / (s if s > 0 else 1.0)
        if e > worst:
            worst, where = e, names[v]
    if eq == 1 and dim == 3:
        # Bx = b1 + (a10 + a11) x + a4 y + a5 z, By = b2 + a6 x - a10 y + a7 z,
        # Bz = b3 + a8 x + a9 y - a11 z   (planes b1..b3, a4..a11 after the Taylor ones)
        b0 = nT * K
        dd = np.abs(got[b0:] - ref[b0:])
        hx, hy, hz = 0.5 * h[0], 0.5 * h[1], 0.5 * h[2]
        dbx = dd[0] + (dd[9] + dd[10]) * hx + dd[3] * hy + dd[4] * hz
        dby = dd[1] + dd[5] * hx + dd[9] * hy + dd[6] * hz
        dbz = dd[2] + dd[7] * hx + dd[8] * hy + dd[10] * hz
        r = ref[b0:]
        s = np.sqrt(r[0] ** 2 + r[1] ** 2 + r[2] ** 2).max()
        e = max(dbx.max(), dby.max(), dbz.max()) / (s if s > 0 else 1.0)
        if e > worst:
            worst, where = e, "B"
        return worst, where
    if eq == 1:
        b0 = nT * K
        g, r = got[b0:], ref[b0:]
        dd = np.abs(g - r)
        hx, hy = 0.5 * h[0], 0.5 * h[1]
        # Bx = b1 + a3 x + a1 y,  By = b2 + a2 x - a3 y
        dbx = dd[0] + dd[4] * hx + dd[2] * hy
        dby = dd[1] + dd[3] * hx + dd[4] * hy
        s = np.sqrt(r[0] ** 2 + r[1] ** 2).max()
        e = max(dbx.max(), dby.max()) / (s if s > 0 else 1.0)
        if e > worst:
            worst, where = e, "B"
    return worst, where


def coef_classes(eq, dim):
    """Groups of interchange planes: (variable, average) and (variable, derivatives)."""
    nT = 4 if dim == 2 else 5
    groups = []
    for v in range(nT):
        groups.append([v * (dim + 1)])
        groups.append(list(range(v * (dim + 1) + 1, (v + 1) * (dim + 1))))
    if eq == 1:
        b0 = nT * (dim + 1)
        groups.append([b0, b0 + 1])
        groups.append([b0 + 2, b0 + 3, b0 + 4])
    return groups


def class_rel_err(got, ref, eq, dim):
    """max over (variable, coefficient class) of max|got - ref| / max|ref| (reported
    for information; ill-posed for classes that are zero in the reference)."""
    worst, where = 0.0, None
    for g in coef_classes(eq, dim):
        d = np.abs(got[g] - ref[g]).max()
        s = np.abs(ref[g]).max()
        e = d / s if s > 0 else d
        if e > worst:
            worst, where = e, g
    return worst, where


def class_errors(got, ref, eq, dim):
    """[(variable, class, error / the class's own largest |ref|, largest |ref|)] for
    every (variable, coefficient class): the per-class figure that the polynomial
    error above replaces (reported, not a bar)."""
    nT = 4 if dim == 2 else 5
    names = (["rho", "mx", "my", "E"] if dim == 2 else ["rho", "mx", "my", "mz", "E"])
    out = []
    for v in range(nT):
        for cls, planes in (("average", [v * (dim + 1)]),
                            ("derivatives", list(range(v * (dim + 1) + 1, (v + 1) * (dim + 1))))):
            s = np.abs(ref[planes]).max()
            d = np.abs(got[planes] - ref[planes]).max()
            out.append((names[v], cls, d / s if s > 0 else d, s))
    if eq == 1:
        b0 = nT * (dim + 1)
        nb = dim
        nd = 3 if dim == 2 else 8
        for cls, planes in (("average", list(range(b0, b0 + nb))),
                            ("derivatives", list(range(b0 + nb, b0 + nb + nd)))):
            s = np.abs(ref[planes]).max()
            d = np.abs(got[planes] - ref[planes]).max()
            out.append(("B", cls, d / s if s > 0 else d, s))
    return out
