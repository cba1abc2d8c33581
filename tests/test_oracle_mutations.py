"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins
catch every one of them: a wrong sign, a dropped scale, an off-by-one shift,
a wrong window exponent or normalisation, a wrong synthesis scale, a wrong
stream phase or crop, a conjugated carrier, a wrong Kaiser argument, a wrong
frame-amplification formula."""
import math

import numpy as np
import pytest

from oracle import qtam_oracle as O
from tests import test_oracle_pins as pins

PIN_TESTS = [
    lambda gd: pins.test_dense_tile_relation_bruteforce_time_domain(),
    lambda gd: pins.test_round_trip_fp64_is_projection(),
    lambda gd: pins.test_parseval_per_row_and_frame_energy(),
    lambda gd: pins.test_adjoint_dot_product(),
    lambda gd: pins.test_shift_invariance_one_decimation_step(),
    lambda gd: pins.test_tone_peaks_on_its_row(),
    lambda gd: pins.test_window_norms(),
    lambda gd: pins.test_bisquare_shape_and_moments(),
    lambda gd: pins.test_geometry_hand_derivations(gd),
    lambda gd: pins.test_grid_and_widths_follow_formulas(),
    lambda gd: pins.test_stream_of_a_periodic_signal_tiles_the_circular_transform(False),
    lambda gd: pins.test_stream_of_a_periodic_signal_tiles_the_circular_transform(True),
    lambda gd: pins.test_stream_layout_rules(),
    lambda gd: pins.test_remodulated_tile_is_the_unshifted_filtered_spectrum(),
    lambda gd: pins.test_single_tile_inverse_recovers_the_signal(True),
    lambda gd: pins.test_kaiser_window_integral_closed_form(),
    lambda gd: pins.test_kappa_hand_case(),
]


def _fwd_wrong_sign(g, X, p, k):
    d, fb = O.band(g, p, k)
    Z = np.zeros(g.M, dtype=np.complex128)
    Z[d % g.M] = g.c[p, k] * O.bisquare_profile(d, int(g.h[p, k])) * X[fb]
    return np.fft.fft(Z) / g.M * math.sqrt(g.M / g.N)


def _fwd_no_renorm(g, X, p, k):
    d, fb = O.band(g, p, k)
    Z = np.zeros(g.M, dtype=np.complex128)
    Z[d % g.M] = g.c[p, k] * O.bisquare_profile(d, int(g.h[p, k])) * X[fb]
    return np.fft.ifft(Z)


def _fwd_shift_off_by_one(g, X, p, k):
    d, fb = O.band(g, p, k)
    Z = np.zeros(g.M, dtype=np.complex128)
    Z[(d + 1) % g.M] = g.c[p, k] * O.bisquare_profile(d, int(g.h[p, k])) * X[fb]
    return np.fft.ifft(Z) * math.sqrt(g.M / g.N)


_orig_profile = O.bisquare_profile
_orig_norm = O.window_norm
_orig_acc = O.accumulate


def _profile_linear(d, h):
    return np.sqrt(_orig_profile(d, h))


def _norm_sum_not_sqrt(h, norm, *args):
    c = _orig_norm(h, norm, *args)
    return c * c if norm == "l2" else c


def _acc_wrong_scale(g, Y, planes=None):
    return _orig_acc(g, Y, planes) * math.sqrt(g.M / g.N) / math.sqrt(g.N / g.M)


def _acc_conj(g, Y, planes=None):
    return _orig_acc(g, np.conj(Y), planes)


_orig_window_profile = O.window_profile


def _kaiser_argument_without_sqrt(d, h, window="bisquare", param=0.0):
    if window != "kaiser":
        return _orig_window_profile(d, h, window, param)
    u = np.abs(np.asarray(d, dtype=np.float64)) / float(h)
    w = np.i0(float(param) * np.clip(1.0 - u * u, 0.0, None)) / np.i0(float(param))
    return np.where(u <= 1.0, w, 0.0)


_orig_kappa = O.kappa


def _kappa_of_squared_windows(g, planes=None, tau=0.0):
    # max W^2 / P instead of max W / P
    planes = range(g.P) if planes is None else planes
    Pf = O.frame_operator(g, planes)
    Wmax = np.zeros(g.Nr)
    for p in planes:
        for k in range(g.K):
            Wmax = np.maximum(Wmax, O.window(g, p, k))
    keep = O.kept_bins(Pf, tau)
    return float(np.max(Wmax[keep] ** 2 / Pf[keep]))


_orig_carrier = O.carrier


def _carrier_conj(g, p, k):
    return np.conj(_orig_carrier(g, p, k))


_orig_phase = O.stream_phase
_orig_layout = O.stream_layout


def _phase_wrong_sign(g, a):
    return np.conj(_orig_phase(g, a))


def _phase_on_remodulated_tiles(g, a):
    m = np.mod(g.kc.astype(np.int64) * int(a), g.N)
    return np.exp(-2j * np.pi * m / g.N)     # the demodulated tiles' factor, whatever the plan


def _layout_crop_off_by_one(g, hop):
    G, Hn, Gm = _orig_layout(g, hop)
    return G, Hn, Gm + 1


MUTANTS = {
    "ifft sign": ("forward_row", _fwd_wrong_sign),
    "dropped sqrt(M/N)": ("forward_row", _fwd_no_renorm),
    "baseband shift off by one": ("forward_row", _fwd_shift_off_by_one),
    "window exponent 1": ("bisquare_profile", _profile_linear),
    "c_k squared": ("window_norm", _norm_sum_not_sqrt),
    "synthesis scale sqrt(M/N)": ("accumulate", _acc_wrong_scale),
    "synthesis of conj(Y)": ("accumulate", _acc_conj),
    "stream phase conjugated": ("stream_phase", _phase_wrong_sign),
    "stream phase on remodulated tiles": ("stream_phase", _phase_on_remodulated_tiles),
    "stream crop one column late": ("stream_layout", _layout_crop_off_by_one),
    "remodulation with the conjugate carrier": ("carrier", _carrier_conj),
    "Kaiser I0 argument beta (1 - u^2)": ("window_profile", _kaiser_argument_without_sqrt),
    "kappa of squared windows": ("kappa", _kappa_of_squared_windows),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, monkeypatch, golden_dir):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(O, attr, fn)
    caught = []
    for t in PIN_TESTS:
        try:
            t(golden_dir)
        except (AssertionError, ValueError, IndexError):
            caught.append(t)
    assert caught, f"no pin caught the mutant '{name}'"
