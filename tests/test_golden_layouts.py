"""The brickwork bond layout reproduces the parameter counts the paper prints."""
import os

from workloads import generators as gen

HERE = os.path.dirname(os.path.abspath(__file__))


def test_brickwork_bond_counts_match_paper():
    rows = []
    with open(os.path.join(HERE, "golden", "paper_layout_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, L, P = (int(v) for v in line.split()[:3])
                rows.append((n, L, P))
    assert len(rows) == 4
    for n, L, P in rows:
        per_layer = len(gen.brickwork_bonds(n, 0)) + len(gen.brickwork_bonds(n, 1))
        assert 15 * L * per_layer == P
