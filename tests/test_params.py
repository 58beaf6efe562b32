"""LM parameter validation on the host (pget_check_params, run first by every call that
takes parameters), on the CPU.

- the library defaults pass;
- each field's bad values are refused with a message naming the field: NaN, out of range,
  inconsistent pairs, unknown enums;
- random parameter sets, including extreme and non-finite values, are either refused or
  satisfy every documented constraint; validation never crashes.
"""
import math

import pytest

from paper_2604_26745_gb300 import pget as P

NAN, INF = float("nan"), float("inf")

BAD = [
    ("max_iters", -1), ("cg_max_iters", -1),
    ("lambda_max", 0.0), ("lambda_max", NAN), ("mu_max", -1.0),
    ("alpha_lambda", -1e-3), ("alpha_mu", NAN),
    ("tv_eps", NAN), ("tv_eps", INF),
    ("cg_rel_tol", NAN),
    ("nu0_scale", 0.0), ("nu0_scale", INF), ("nu0_scale", NAN),
    ("nu_up", 0.5), ("nu_down", 0.0), ("nu_down", 2.0),
    ("eta", NAN), ("rho_lo", 0.9), ("rho_hi", INF),
    ("nu_min", 0.0), ("nu_max", 1e-13), ("nu_min", NAN),
    ("precision", 4), ("precision", -1), ("alpha_decay", 0.5), ("alpha_decay_iters", -1),
    ("inner_solver", 2), ("lin_constraint", 2),
]


def test_defaults_pass():
    P.check_params(P.default_params())
    P.check_params(P.default_params(tv_eps=-1.0, alpha_decay=5.0, alpha_decay_iters=3, inner_solver=1,
                                    lin_constraint=1, lin_slope=10.0, lin_offset=0.1, precision=P.PGET_F64))


@pytest.mark.parametrize("field,value", BAD)
def test_bad_values_are_refused(field, value):
    p = P.default_params()
    setattr(p, field, value)
    with pytest.raises(ValueError, match="invalid parameters"):
        P.check_params(p)


@pytest.mark.parametrize("kw", [dict(lin_slope=-1.0), dict(lin_slope=NAN), dict(lin_offset=-0.1),
                                dict(lin_offset=INF)])
def test_bad_linear_bounds_are_refused(kw):
    p = P.default_params(lin_constraint=1, **{"lin_slope": 1.0, "lin_offset": 0.0, **kw})
    with pytest.raises(ValueError, match="linear bound"):
        P.check_params(p)


try:  # the property test needs hypothesis; the tests above run without it
    import hypothesis as hyp
    from hypothesis import strategies as st
except ImportError:  # pragma: no cover
    hyp = None

if hyp is not None:
    reals = st.one_of(st.floats(allow_nan=True, allow_infinity=True, width=64),
                      st.sampled_from([0.0, 1e-12, 0.25, 0.75, 1.0, 4.0, 1e12, -1.0]))


    @hyp.settings(max_examples=300, deadline=None, derandomize=True)
    @hyp.given(f=st.fixed_dictionaries({k: reals for k in (
        "lambda_max", "mu_max", "alpha_lambda", "alpha_mu", "tv_eps", "cg_rel_tol", "nu0_scale", "nu_up", "nu_down",
        "eta", "rho_lo", "rho_hi", "nu_min", "nu_max", "alpha_decay")}),
        i=st.fixed_dictionaries({"max_iters": st.integers(-2, 50), "cg_max_iters": st.integers(-2, 50),
                                 "precision": st.integers(-1, 4), "alpha_decay_iters": st.integers(-2, 5),
                                 "inner_solver": st.integers(-1, 2)}))
    def test_random_parameters_are_refused_or_consistent(f, i):
        p = P.default_params()
        for k, v in {**f, **i}.items():
            setattr(p, k, v)
        try:
            P.check_params(p)
        except ValueError:
            return
        assert p.max_iters >= 0 and p.cg_max_iters >= 0 and p.precision in (0, 1, 2, 3) and p.inner_solver in (0, 1)
        assert p.lambda_max > 0 and p.mu_max > 0 and p.alpha_lambda >= 0 and p.alpha_mu >= 0
        assert math.isfinite(p.tv_eps) and not math.isnan(p.cg_rel_tol)
        assert 0 < p.nu0_scale < INF and p.nu_up >= 1 and 0 < p.nu_down <= 1
        assert all(map(math.isfinite, (p.eta, p.rho_lo, p.rho_hi))) and p.rho_lo <= p.rho_hi
        assert 0 < p.nu_min <= p.nu_max
        assert (p.alpha_decay == 0 or p.alpha_decay >= 1) and p.alpha_decay_iters >= 0
