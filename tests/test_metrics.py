"""Front measures on exported fields (host side): a solid block of known size."""
import numpy as np

from paper_2603_22902_gb300.metrics import front_height, front_integral


def block_fields(nx=64, ny=32, w=20, h=7.0):
    phi0 = np.zeros((ny, nx))
    phi0[:16] = 1.0                                # the freezing liquid fills y < 16
    fl = np.ones((ny, nx))
    x0 = nx // 2 - w // 2
    fl[: int(h), x0:x0 + w] = 0.0                  # solid block of height floor(h) on the wall
    fl[int(h), x0:x0 + w] = 1.0 - (h - int(h))     # partly frozen top row
    return {"phi": np.stack([phi0, 1.0 - phi0]), "fl": fl}


def test_front_height_is_the_centre_line_solid_height():
    F = block_fields(h=7.25)
    assert abs(front_height(F, 64) - 7.25) < 1e-12


def test_front_integral_is_the_width_averaged_solid_height():
    F = block_fields(w=20, h=7.25)
    assert abs(front_integral(F, 64) - 7.25 * 20 / 64) < 1e-12
    # the ambient phase never counts, even where f_s = 1
    F["fl"][20:24] = 0.0
    assert abs(front_integral(F, 64) - 7.25 * 20 / 64) < 1e-12
