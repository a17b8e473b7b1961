"""Host pieces of paper_2105_08772_gb300.studies."""
import pytest

St = pytest.importorskip("paper_2105_08772_gb300.studies")


@pytest.mark.parametrize("a,b,R", [(1.0, 4.0, 1.0), (2.0, 3.0, 1.5), (0.5, 1.0, 2.0)])
def test_cs_critical_point_matches_oracle(a, b, R):
    """Closed-form reduction (g(q) = q g'(q)) against the oracle's 2-D root solve of
    dp/dn = d^2p/dn^2 = 0."""
    from oracle import eos as E
    n_c, T_c = St.cs_critical_point(a, b, R)
    rn, rT = E.cs_critical_temperature(E.EOS("cs", a=a, b=b, R=R))
    assert n_c == pytest.approx(rn, rel=1e-8) and T_c == pytest.approx(rT, rel=1e-10)
