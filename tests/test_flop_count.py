"""The FP32 flops per cell-step that bench.py reports (its FP32 view of the
roofline) follow from the method: one cell-step of eq. (3) in face form,
with the two face fluxes a cell owns (east and north) and its own cross
terms evaluated once, counted operation by operation with a float that
tallies its arithmetic (a fused multiply-add would count 2, as a separate
multiply and add do here)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class Counted(float):
    ops = 0

    def _wrap(self, v):
        Counted.ops += 1
        return Counted(v)

    def __add__(self, o): return self._wrap(float(self) + float(o))
    def __radd__(self, o): return self._wrap(float(o) + float(self))
    def __sub__(self, o): return self._wrap(float(self) - float(o))
    def __rsub__(self, o): return self._wrap(float(o) - float(self))
    def __mul__(self, o): return self._wrap(float(self) * float(o))
    def __rmul__(self, o): return self._wrap(float(o) * float(self))
    def __truediv__(self, o): return self._wrap(float(self) / float(o))


def one_cell_step(kahan):
    """Arithmetic that one interior cell performs in one step when every
    face flux is evaluated once (the cell owns its east and north faces; the
    west and south ones are its neighbours' east and north faces)."""
    c = lambda x: Counted(x)
    u, v, w, uE, vE, wE, uN, vN, wN = (c(x) for x in (0.3, 0.4, 0.2, 0.31, 0.42, 0.21, 0.29, 0.38, 0.19))
    wNb, wSb, wEb, wWb = c(0.18), c(0.22), c(0.23), c(0.17)  # tangential neighbours of w
    a11, a11E, a22, a22N, a12, a12N = (c(x) for x in (1.0, 0.9, 0.8, 0.7, 0.1, 0.12))
    zE, zN = c(0.01), c(0.02)  # the neighbours' cross terms (computed by them)
    ihx2, ihy2, kx, ky, kc = (c(x) for x in (4.0, 4.0, 2.0, 2.0, 1.0))
    dt, D, delta, rho, cc = (c(x) for x in (1e-3, 1e-3, 12.5, 1.0, 70.0))
    hW, hS, gW, gS = c(0.0), c(0.0), c(0.0), c(0.0)  # the neighbours' faces
    # tumour faces (Table 1): mobility, difference, product, 1/h^2
    hE = (1 - 0.5 * (u + uE)) * (vE - v) * ihx2
    hN = (1 - 0.5 * (u + uN)) * (vN - v) * ihy2
    # the cell's cross terms (Table 2): tangential differences and products
    zx = a12 * (wNb - wSb)
    zy = a12 * (wEb - wWb)
    # acid faces: mean weight, normal difference and product, the two cells'
    # cross terms summed and weighted, the sum
    gE = (a11 + a11E) * kx * (wE - w) + (zx + zE) * kc
    gN = (a22 + a22N) * ky * (wN - w) + (zy + zN) * kc
    d1 = (hE - hW) + (hN - hS)
    d2 = (gE - gW) + (gN - gS)
    fu = u * (1 - u) - delta * u * w
    fv = rho * v * (1 - v) + D * d1
    fw = cc * (v - w) + d2
    if kahan:
        for x, f, comp in ((u, fu, c(0.0)), (v, fv, c(0.0)), (w, fw, c(0.0))):
            y = dt * f - comp
            t = x + y
            (t - x) - y
    else:
        for x, f in ((u, fu), (v, fv), (w, fw)):
            x + dt * f


def test_flops_per_cell_step_match_bench():
    sys.path.insert(0, ROOT)
    import bench
    for kahan, key in ((False, "fp32"), (True, "fp32_kahan")):
        Counted.ops = 0
        one_cell_step(kahan)
        assert Counted.ops == bench.FLOPS_PER_CELL_STEP[key], (key, Counted.ops)
