"""The tile forward's interior-batch test, emulated in float32 on the CPU.

The forward kernel walks each ray's bands in batches of four and skips the
per-band bounds tests when the pixels of the batch's two end points lie at
least one pixel inside the image.  This checks, over every ray of several
geometries and every band-chunk count, that no band of an admitted batch has
a piece outside the image, i.e. that the unchecked offsets stay in bounds.

The view parameters, the band range and the band points are recomputed here
the way the library computes them (FP64 on the host, rounded to FP32; the
band point is two fused multiply-adds, emulated by an FP64 product and sum
rounded once to FP32, which can differ from a true fma by one ulp in rare
ties -- far inside the one-pixel margin the test keeps).
"""
import math

import numpy as np
import pytest

f32 = np.float32


def _fma(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(f32)


def _snap(x):
    if abs(x) < 1e-12:
        return 0.0
    if abs(abs(x) - 1.0) < 1e-12:
        return math.copysign(1.0, x)
    return x


def _band_point(du, du_lo, uf, kc):
    return _fma(kc, du, _fma(kc, du_lo, uf))


def _admitted_out_of_bounds(nx, ny, na, nb, pixel_mm=2.0, bin_mm=None, chunk_counts=(8, 16, 32)):
    ds = bin_mm or pixel_mm
    bad = admitted = 0
    for i in range(na):
        th = i * math.pi / na
        c, s = _snap(math.cos(th)), _snap(math.sin(th))
        col = abs(c) < abs(s)
        cm, cn = (s, c) if col else (c, s)
        n_minor, n_major = (ny, nx) if col else (nx, ny)
        du64 = -cn / cm
        du = f32(du64)
        du_lo = f32(du64 - float(du))
        inv_du = f32(-cm / cn) if cn != 0.0 else f32(0.0)
        off = 0.5 if n_minor % 2 else 0.0
        sj = (np.arange(nb) - 0.5 * (nb - 1)) * ds
        u = sj / (cm * pixel_mm) + off
        ui_f = np.rint(u)
        ux, uy = ui_f.astype(f32), (u - ui_f).astype(f32)
        mo, hm = n_minor >> 1, f32(0.5 * n_major)
        # band range (a superset of the bands where the ray meets the image)
        uc = (ux + uy).astype(f32)
        if du == 0.0:
            inside = (uc >= f32(-mo)) & (uc < f32(n_minor - mo))
            k_lo = np.zeros(nb, np.int64)
            k_hi = np.where(inside, n_major, 0)
        else:
            ka = _fma((f32(-mo - 1) - uc).astype(f32), inv_du, hm)
            kb = _fma((f32(n_minor - mo + 1) - uc).astype(f32), inv_du, hm)
            kmax = f32(n_major + 1)
            lo = np.minimum(np.maximum(np.minimum(ka, kb), f32(-1)), kmax)
            hi = np.maximum(np.minimum(np.maximum(ka, kb), kmax), f32(-1))
            k_lo = np.maximum(0, np.floor(lo).astype(np.int64) - 1)
            k_hi = np.minimum(n_major, np.ceil(hi).astype(np.int64) + 1)
        ui = ux.astype(np.int64) + (n_minor >> 1)
        for chunks in chunk_counts:
            per = (n_major + chunks - 1) // chunks
            for ch in range(chunks):
                kb_ = np.maximum(k_lo, ch * per)
                ke_ = np.minimum(k_hi, (ch + 1) * per)
                for start in range(0, per, 4):
                    k = kb_ + start
                    live = k < ke_
                    if not live.any():
                        continue
                    kc = (k.astype(f32) - hm).astype(f32)
                    va = _band_point(du, du_lo, uy, kc)
                    vend = _band_point(du, du_lo, uy, (kc + f32(4)).astype(f32))
                    e_lo = np.floor(np.minimum(va, vend)).astype(np.int64) + ui
                    e_hi = np.floor(np.maximum(va, vend)).astype(np.int64) + ui
                    inner = live & (k + 4 <= ke_) & (e_lo >= 1) & (e_hi <= n_minor - 3)
                    admitted += int(inner.sum()) * 4
                    for b in range(4):
                        kc = (kc + f32(1)).astype(f32)
                        vb = _band_point(du, du_lo, uy, kc)
                        m0 = np.floor(np.minimum(va, vb)).astype(np.int64) + ui
                        bad += int((inner & ((m0 < 0) | (m0 > n_minor - 2))).sum())
                        va = vb
    return bad, admitted


@pytest.mark.parametrize("geom", [
    (64, 64, 60, 91),                     # small benchmark image
    (37, 29, 23, 41, 1.7, 1.3),           # odd, non-square, bins != pixels
    (128, 128, 90, 183),
    (96, 80, 37, 131, 2.0, 1.6),          # odd view count, no axis-aligned views but 0
    (256, 256, 180, 367),                 # the benchmark image
])
def test_interior_batches_stay_inside_the_image(geom):
    bad, admitted = _admitted_out_of_bounds(*geom)
    assert admitted > 0
    assert bad == 0


@pytest.mark.slow
def test_interior_batches_stay_inside_the_largest_image():
    """512x512, 720 views x 733 bins (the largest serving size), at the chunk
    counts its launches use."""
    bad, admitted = _admitted_out_of_bounds(512, 512, 720, 733, chunk_counts=(16, 32))
    assert admitted > 0
    assert bad == 0
