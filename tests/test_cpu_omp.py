"""The multi-core CPU CG used as a timing comparison (oracle/fe_cpu_omp.c)
solves the same systems as the serial oracle, in both storage forms."""
import numpy as np
import pytest

import fe_inputs
import oracle


@pytest.mark.parametrize("dims", [(9, 9, 9), (7, 5, 11)])
def test_omp_cg_matches_oracle(dims):
    face = fe_inputs.face_data(11, 0, *dims)
    s = oracle.build_system(*dims, face)
    x, it, rel, st = oracle.cg(s["row_ptr"], s["cols"], s["vals"], s["b"], tol=1e-12, maxit=2000)
    ptr, jas, off = oracle.csr_to_bcrs(s["row_ptr"], s["cols"])
    runs = [oracle.omp_cg("csr", s["b"], s["row_ptr"], s["cols"], s["vals"], tol=1e-12, maxit=2000),
            oracle.omp_cg("bcrs", s["b"], ptr, jas, s["vals"], offsets=off, tol=1e-12, maxit=2000)]
    assert st == oracle.CG_CONVERGED
    for xo, ito, relo, sto, sec, thr in runs:
        assert sto == oracle.CG_CONVERGED and abs(ito - it) <= 1 and thr >= 1 and sec >= 0.0
        assert np.linalg.norm(xo - x) <= 1e-10 * np.linalg.norm(x)
        assert oracle.true_relres(s["row_ptr"], s["cols"], s["vals"], s["b"], xo) <= 1.5e-12


def test_omp_cg_zero_rhs_and_maxit():
    s = oracle.build_system(5, 5, 5)
    xo, it, rel, st, _, _ = oracle.omp_cg("csr", np.zeros_like(s["b"]), s["row_ptr"], s["cols"],
                                          s["vals"], x0=np.ones_like(s["b"]))
    assert st == oracle.CG_CONVERGED and it == 0 and not xo.any()
    xo, it, rel, st, _, _ = oracle.omp_cg("csr", s["b"], s["row_ptr"], s["cols"], s["vals"],
                                          tol=1e-14, maxit=3)
    assert st == oracle.CG_MAXIT and it == 3
