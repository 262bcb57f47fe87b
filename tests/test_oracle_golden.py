"""Golden values printed in the paper: the parameter table of Sec. 6 (tab:ALL-params)."""
import math
import os

from oracle import scheme as S

HERE = os.path.dirname(os.path.abspath(__file__))


def _rows():
    with open(os.path.join(HERE, "golden", "paper_params_table.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                run, n, M, c, alpha, beta, kxi, dxxi, xi, nv = line.split()
                yield run, int(n), float(M), float(c), float(alpha), float(beta), float(kxi), float(dxxi), float(xi), int(nv)


def test_parameter_table_is_reproduced():
    rows = list(_rows())
    assert len(rows) == 4
    for run, n, M, c, alpha, beta, kxi, dxxi, xi, nv in rows:
        p = S.Params(n, alpha, 2.0 / alpha, 1e-3)    # alpha beta = 1/(2 M^2) = 2 (eq-scaling-choice3)
        assert abs(p.beta - beta) < 1e-9, run
        assert abs(p.xi - xi) < 5e-7, run            # xi = sqrt(alpha/beta), printed to 6 decimals
        q = S.params_from_xi(n, p.xi, 1e-3)          # and back: alpha = sqrt(2) xi
        assert abs(q.alpha - alpha) < 1e-15 and abs(q.beta - beta) < 1e-9, run
        assert abs(math.sqrt(2 * p.alpha * p.beta) - c) < 1e-12, run        # c = sqrt(2 alpha beta)
        assert abs(1.0 / math.sqrt(2 * p.alpha * p.beta) - M) < 1e-12, run  # M = 1/c
        assert abs((n / 2) * p.xi - kxi) < 5e-3, run                         # k_max xi, L = 2 pi
        assert abs(p.dx / p.xi - dxxi) < 5e-4, run
        assert int(2 * math.pi / (2 * p.xi)) == nv, run                      # Nv1d = L / (2 xi)
