"""The FP32-mixed push flushes its shared-memory deposit tile quad by quad and turns a flat quad
index into (grid, plane, row, quad) with FP32 products by approximate reciprocals (the kernel's
`__fdividef`, at most 2 ulp).  For every tile shape that fits the 4096-entry tile (rows of whole
quads, three or four grids), every index must decode to the integer quotients even when the
reciprocal is off by 2^-21 relative either way (4x the documented bound) and the product rounds
the same way: the index arithmetic the kernel relies on, checked on the host."""
import numpy as np

TILE = 4096
f32 = np.float32


def _quot(i, d, e):
    r = f32(f32(1.0) / f32(d)) * f32(1.0 + e)
    p = (i.astype(np.float32) + f32(0.5)) * r
    return np.floor(p * f32(1.0 + np.sign(e) * 2.0 ** -24)).astype(np.int64)


def test_every_tile_shape_decodes_exactly():
    shapes = 0
    for ngrid in (3, 4):
        for tx in range(4, TILE, 4):
            for ty in range(1, TILE):
                if ngrid * tx * ty + 4 > TILE:
                    break
                for tz in range(1, TILE):
                    vol = tx * ty * tz
                    if ngrid * vol + 4 > TILE:
                        break
                    shapes += 1
                    qx, vq = tx // 4, vol // 4
                    i = np.arange(ngrid * vq, dtype=np.int64)
                    c = i // vq
                    r = i - c * vq
                    k = r // (qx * ty)
                    j = (r - k * qx * ty) // qx
                    for e in (-2.0 ** -21, 2.0 ** -21):
                        c2 = _quot(i, vq, e)
                        r2 = i - c2 * vq
                        k2 = _quot(r2, qx * ty, e)
                        j2 = _quot(r2 - k2 * qx * ty, qx, e)
                        assert np.array_equal(c2, c) and np.array_equal(k2, k) and np.array_equal(j2, j), (
                            ngrid, tx, ty, tz, e)
    assert shapes > 10000
