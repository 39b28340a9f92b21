"""The seeded input generator: C implementation vs its numpy restatement,
determinism, and the porosity stopping rule."""
import numpy as np
import pytest

import lbm_inputs


def test_splitmix64_published_values():
    # splitmix64 from state 0: the first outputs of the published generator
    # (Steele, Lea, Flood 2014; the seeding routine of xoshiro by Vigna).
    out = lbm_inputs.splitmix64(0, 3)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


@pytest.mark.parametrize("dims,r,phi,seed", [((12, 10, 9), 2.5, 0.7, 1), ((16, 16, 16), 3.0, 0.5, 2),
                                             ((7, 9, 11), 4.2, 0.85, 3), ((5, 5, 5), 6.0, 0.3, 4)])
def test_sphere_pack_c_matches_numpy(dims, r, phi, seed):
    nx, ny, nz = dims
    a, ia = lbm_inputs.sphere_pack(nx, ny, nz, r, phi, seed)
    b, ib = lbm_inputs.sphere_pack_numpy(nx, ny, nz, r, phi, seed)
    assert np.array_equal(a, b)
    assert ia == ib
    assert ia.porosity <= phi
    assert ia.porosity == pytest.approx(1 - a.mean())


def test_sphere_pack_stops_at_first_crossing():
    m, info = lbm_inputs.sphere_pack(20, 20, 20, 3.0, 0.8, 9)
    prev, pinfo = lbm_inputs.sphere_pack(20, 20, 20, 3.0, 0.0, 9, max_spheres=info.spheres - 1)
    assert pinfo.porosity > 0.8 >= info.porosity
    assert np.all(m >= prev)


def test_channel_and_fields():
    m = lbm_inputs.channel(4, 3, 8)
    assert m.shape == (8, 3, 4) and m[0].all() and m[7].all() and not m[1:7].any()
    f1 = lbm_inputs.random_fields((3, 4, 5), 7, 1e-3, 2e-3, None)
    f2 = lbm_inputs.random_fields((3, 4, 5), 7, 1e-3, 2e-3, None)
    assert all(np.array_equal(x, y) for x, y in zip(f1, f2))
    assert np.abs(f1[0]).max() <= 1e-3 and np.abs(f1[1]).max() <= 2e-3
