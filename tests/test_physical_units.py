"""The physical-unit front end (Eq. 2's optics: wavelength, focal length,
pixel pitch) maps spots in metres to the normalised units of every solve.
Pinned to optics, not to its own formula: the first diffraction order of the
P-pixel aperture is one cycle across it, and the axial shift of a focus
equals, for small shifts, the paraxial quadratic phase that a thin lens adds.
Host-only calls: no GPU."""
import math

import numpy as np
import pytest

# the paper's optics (Section 4): 800 nm, 9.2 um pixels, a 1152-pixel aperture;
# the focal length is not printed, 200 mm is taken as an example
LAM, F, PITCH, P = 800e-9, 0.2, 9.2e-6, 1152


def _conv(xyz, P=P, lam=LAM, f=F, pitch=PITCH):
    from paper_2003_05293_gb300 import spots_from_physical
    return spots_from_physical(xyz, P, lam, f, pitch)


def test_first_diffraction_order_is_one_cycle():
    # a grating of period D = P pitch diffracts its first order to sin(t) = lam / D,
    # i.e. to x = f lam / D in the focal plane: alpha = 1 there (beta likewise)
    x1 = F * LAM / (P * PITCH)
    s = _conv(np.array([[x1, 0.0, 0.0], [0.0, -2.5 * x1, 0.0], [7.25 * x1, 3 * x1, 0.0]]))
    assert s[0] == pytest.approx([1.0, 0.0, 0.0], abs=1e-12)
    assert s[1] == pytest.approx([0.0, -2.5, 0.0], abs=1e-12)
    assert s[2] == pytest.approx([7.25, 3.0, 0.0], abs=1e-12)


@pytest.mark.parametrize("z", [1e-6, 10e-6, -25e-6])
def test_defocus_is_the_paraxial_lens_phase(z):
    # moving the focus of a lens of focal length f to f + z takes an added thin
    # lens of power 1/f - 1/(f + z); its phase pi rho^2 (1/f - 1/(f+z)) / lam at
    # the aperture edge, in waves, is gamma to first order in z / f
    edge = P * PITCH / 2
    exact = edge ** 2 * (1 / F - 1 / (F + z)) / (2 * LAM)
    g = _conv(np.array([[0.0, 0.0, z]]))[0, 2]
    assert g == pytest.approx(exact, rel=5 * abs(z) / F)
    assert math.copysign(1, g) == math.copysign(1, z)


def test_linear_and_in_place():
    from paper_2003_05293_gb300 import capi
    import ctypes
    rng = np.random.default_rng(0)
    a = rng.normal(0, 1e-4, (5, 3))
    b = rng.normal(0, 1e-4, (5, 3))
    assert np.allclose(_conv(a + 2 * b), _conv(a) + 2 * _conv(b), rtol=1e-12, atol=1e-12)
    # in place (the C function allows spots_out == xyz_m)
    lib = capi.load()
    o = capi.cswgs_optics(LAM, F, PITCH)
    buf = a.copy()
    p = buf.ctypes.data_as(capi.c_double_p)
    assert lib.cswgs_spots_from_physical(ctypes.byref(o), p, 5, P, p) == 0
    assert np.allclose(buf, _conv(a), rtol=0, atol=0)


def test_bad_optics_refused():
    from paper_2003_05293_gb300 import CswgsError
    for kw in (dict(lam=0.0), dict(f=-1.0), dict(pitch=float("nan")), dict(P=1)):
        with pytest.raises(CswgsError):
            _conv(np.zeros((1, 3)), **kw)
    with pytest.raises(CswgsError):
        _conv(np.array([[0.0, float("inf"), 0.0]]))
