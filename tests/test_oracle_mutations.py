"""Planted mistakes in the oracle (on the CPU) must fail its pins.

Each test patches one step of the oracle with a plausible mistake (a
transposed operand, a dropped term, a wrong sign) and checks that the pin that
guards that step no longer holds.
"""

import numpy as np
import pytest

import oracle as orc
import oracle.eer4d_oracle as core
from test_oracle_pins import (_lens, _weak_phase_case, test_scan_rotation_direction_from_forward_model,
                              test_spherical_aberration_term_from_forward_model)


def _weak_err(**kw):
    phi, ref, _ = _weak_phase_case(0.01, **kw)
    return np.linalg.norm(phi - ref) / np.linalg.norm(ref), np.corrcoef(phi.ravel(), ref.ravel())[0, 1]


def test_unmutated_baseline():
    err, r = _weak_err(ny=32, nx=16)
    assert err < 1e-3 and r > 0.999


def test_transposed_scan_frequencies_fail(monkeypatch):
    real = core.kprime_f64

    def swapped(geom, rot):
        g = dict(geom, kpm_x=geom["kpm_y"], kpm_y=geom["kpm_x"])
        kx, ky = real(g, rot)
        return kx, ky

    monkeypatch.setattr(core, "kprime_f64", swapped)
    monkeypatch.setattr(core, "kprime_f32", lambda geom, rot: tuple(
        a.astype(np.float32) for a in swapped(geom, rot)))
    err, _ = _weak_err(ny=32, nx=16)
    assert err > 0.1


def test_other_sideband_fails(monkeypatch):
    real = core.trotter_mask
    monkeypatch.setattr(core, "trotter_mask", lambda kx, ky, KX, KY, k0sq: real(kx, ky, -KX, -KY, k0sq))
    _, r = _weak_err()
    assert r < 0


def test_conjugate_aberration_correction_fails(monkeypatch):
    real = core.chi_turns
    monkeypatch.setattr(core, "chi_turns", lambda qx, qy, ab, g: -real(qx, qy, ab, g))
    _, r = _weak_err(aberr=(80.0, 20.0, -15.0, 0.0, 0.0))
    assert r < 0.9


def test_dropped_astigmatism_term_fails(monkeypatch):
    real = core.chi_turns
    monkeypatch.setattr(core, "chi_turns", lambda qx, qy, ab, g: real(qx, qy, (ab[0], ab[1], 0.0, ab[3]), g))
    _, r = _weak_err(aberr=(0.0, 0.0, 100.0, 0.0, 0.0))
    assert r < 0.98  # the aberration pin requires r > 0.98 with the true aberrations


def test_dropped_exclusion_disk_fails(monkeypatch):
    def lens_only(kx, ky, KX, KY, k0sq):
        f = np.float32
        dxm, dym = f(kx) - KX, f(ky) - KY
        return (dxm * dxm + dym * dym) < k0sq

    monkeypatch.setattr(core, "trotter_mask", lens_only)
    import synth
    w = synth.workload(2, scan_ny=64, scan_nx=64)
    geom = synth.geometry(w)
    G = np.ones((orc.pixel_table(geom)["P"], 64, 64), dtype=np.complex128)
    _, nK = orc.ssb_spectrum(G, geom, (0, 0, 0, 0, 0))
    KX, KY = orc.kprime_f64(geom, 0.0)
    s = np.hypot(KX, KY)
    area = _lens(s, geom["k0_px"]) - _lens(2 * s, geom["k0_px"])
    assert np.abs(nK - area).max() > 4 * np.pi * geom["k0_px"]


def test_wrong_phase_image_part_fails(monkeypatch):
    real_ifft2 = np.fft.ifft2

    class FakeFFT:
        def __getattr__(self, n):
            return getattr(np.fft, n)

        @staticmethod
        def ifft2(a, *args, **kw):
            out = real_ifft2(a, *args, **kw)
            return out.real + 1j * out.real  # Re taken where Im is meant

    class FakeNP:
        def __getattr__(self, n):
            return getattr(np, n)
        fft = FakeFFT()

    monkeypatch.setattr(core, "np", FakeNP())
    _, r = _weak_err()
    assert abs(r) < 0.5


def test_doubled_spherical_coefficient_fails(monkeypatch):
    """C3 w^4/2 in place of C3 w^4/4 (and its derivative) fails the C3 pin."""
    real = core.chi_turns
    monkeypatch.setattr(core, "chi_turns",
                        lambda qx, qy, ab, g: real(qx, qy, ab, g) + real(qx, qy, (0.0, 0.0, 0.0, ab[3]), g))
    with pytest.raises(AssertionError):
        test_spherical_aberration_term_from_forward_model()


def test_spherical_term_sign_fails(monkeypatch):
    real = core.chi_turns
    monkeypatch.setattr(core, "chi_turns",
                        lambda qx, qy, ab, g: real(qx, qy, (ab[0], ab[1], ab[2], -ab[3]), g))
    with pytest.raises(AssertionError):
        test_spherical_aberration_term_from_forward_model()


def test_rotation_sign_flipped_consistently_fails(monkeypatch):
    """K' = R(-rot) K in every place the oracle forms K' (the float32 mask
    and the double phase) fails the rotation pin."""
    r32, r64 = core.kprime_f32, core.kprime_f64
    monkeypatch.setattr(core, "kprime_f32", lambda geom, rot: r32(geom, -rot))
    monkeypatch.setattr(core, "kprime_f64", lambda geom, rot: r64(geom, -rot))
    with pytest.raises(AssertionError):
        test_scan_rotation_direction_from_forward_model()
