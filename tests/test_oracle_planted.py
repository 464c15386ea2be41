"""Planted mistakes in the oracle, on the CPU.  Each plausible error is
patched into the oracle for one test, and at least one of the oracle's pins
must then fail.  The errors: a lost normalization, a Condon-Shortley sign, a
perturbed recurrence coefficient, weights or nodes that are slightly off, an
analysis without weights, a phi synthesis without the factor 2 of +-m, a phi
analysis without its conjugate, and an adjoint carrying weights.  This shows
that the pins constrain what they are meant to."""

import numpy as np
import pytest

import oracle
import oracle.legendre as OL
import oracle.sht as OS

import tests.test_oracle_legendre as TL
import tests.test_oracle_quadrature as TQ
import tests.test_oracle_sht as TS

PINS = [
    ("closed forms", lambda: TL.test_closed_forms()),
    ("definition, k = 5", lambda: TL.test_matches_definition_exactly_for_low_degrees(5)),
    ("Unsold sum", lambda: TL.test_unsold_sum(6)),
    ("addition theorem", lambda: TL.test_addition_theorem(10)),
    ("orthonormal on the interval", lambda: TL.test_orthonormal_on_interval()),
    ("parity", lambda: TL.test_parity()),
    ("numpy leggauss", lambda: TQ.test_nodes_match_numpy_leggauss(17)),
    ("zeros and exactness", lambda: TQ.test_nodes_are_zeros_of_P2l_and_rule_is_exact(4)),
    ("paper weights at m = 0", lambda: TQ.test_paper_weights_at_m0_equal_twice_gl_weights(8)),
    ("brute force", lambda: TS.test_brute_force_synthesis(2)),
    ("round trip", lambda: TS.test_round_trip(3)),
    ("special fields", lambda: TS.test_special_fields()),
    ("phi stage vs numpy fft", lambda: TS.test_phi_stage_against_numpy_fft()),
    ("single mode", lambda: TS.test_single_mode()),
    ("weighted adjoint", lambda: TS.test_analysis_is_weighted_adjoint()),
]

_table = OL.legendre_table
_nodes = OL.gl_nodes_weights
_adjoint = OS.legendre_adjoint
_phase = OS._phase_matrix


def _lost_normalization(m, x, kmax):
    return np.sqrt(2.0) * _table(m, x, kmax)


def _condon_shortley(m, x, kmax):
    return (-1.0) ** m * _table(m, x, kmax)


def _perturbed_coefficient(m, x, kmax):
    t = _table(m, x, kmax)
    return t * (1.0 + 1e-9 * np.arange(t.shape[0]))[:, None]


def _weights_off(npts):
    x, w = _nodes(npts)
    return x, w * (1.0 + 1e-9)


def _nodes_off(npts):
    x, w = _nodes(npts)
    return x + 1e-12 * np.sign(x), w


def _analysis_without_weights(G, l, orders=None):
    return _adjoint(G, l, orders)


def _phi_synthesis_without_factor_2(G, l):
    return np.real(np.asarray(G, dtype=np.complex128).T @ _phase(l))


def _phi_analysis_without_conjugate(f, l):
    return (_phase(l) @ np.asarray(f, dtype=np.float64).T) / (4 * int(l) - 1)


def _adjoint_with_weights(Ghat, l, orders=None):
    _, w = _nodes(2 * int(l))
    return _adjoint(np.asarray(Ghat) * w, l, orders)


MUTANTS = {
    "lost 1/sqrt(2) normalization": ("legendre_table", _lost_normalization),
    "Condon-Shortley sign": ("legendre_table", _condon_shortley),
    "perturbed recurrence coefficient": ("legendre_table", _perturbed_coefficient),
    "weights off by 1e-9": ("gl_nodes_weights", _weights_off),
    "nodes off by 1e-12": ("gl_nodes_weights", _nodes_off),
    "analysis without weights": ("legendre_analysis", _analysis_without_weights),
    "phi synthesis without the factor 2": ("phi_synthesis", _phi_synthesis_without_factor_2),
    "phi analysis without the conjugate": ("phi_analysis", _phi_analysis_without_conjugate),
    "adjoint with weights": ("legendre_adjoint", _adjoint_with_weights),
}


def _failing_pins():
    failed = []
    for name, pin in PINS:
        try:
            pin()
        except AssertionError:
            failed.append(name)
    return failed


def test_every_pin_passes_on_the_oracle_as_it_stands():
    assert _failing_pins() == []


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_a_planted_mistake_fails_a_pin(monkeypatch, mutant):
    name, fn = MUTANTS[mutant]
    for mod in (oracle, OL, OS):
        if hasattr(mod, name):
            monkeypatch.setattr(mod, name, fn)
    assert _failing_pins(), mutant
