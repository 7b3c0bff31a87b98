"""The seeded input generators: geometry conventions and determinism."""
import numpy as np

from paper_2312_15554_gb300 import inputs as I


def test_sphere_pack_reaches_its_porosity_and_is_reproducible():
    H1, c1, r1 = I.sphere_pack((32, 32, 32), 0.4, (3.0, 6.0), 5)
    H2, c2, r2 = I.sphere_pack((32, 32, 32), 0.4, (3.0, 6.0), 5)
    assert np.array_equal(H1, H2)
    assert 1 - H1.mean() <= 0.4 < 1 - H1.mean() + 0.05


def test_dissolution_removes_interface_solid_only():
    H = I.sphere_pack((24, 24, 24), 0.35, 4.0, 3)[0]
    D = I.dissolve(H, 1)
    assert ((D == 1) <= (H == 1)).all()              # nothing turns solid
    removed = (H == 1) & (D == 0)
    pore = H == 0
    touch = np.zeros_like(pore)
    for ax in range(3):
        touch |= np.roll(pore, 1, axis=ax) | np.roll(pore, -1, axis=ax)
    assert (removed == ((H == 1) & touch)).all()    # exactly the solid face-adjacent to pore
    P = I.dissolve(H, 1, fraction=0.3, seed=1)
    assert np.array_equal(P, I.dissolve(H, 1, fraction=0.3, seed=1))
    part = (H == 1) & (P == 0)
    assert (part <= removed).all() and 0.2 < part.sum() / removed.sum() < 0.4
