"""No CPU fallback: every public entry point of the product package, handed
CPU tensors (or run where no GPU is usable), raises instead of computing."""

import pytest
import torch

import paper_2407_19892_gb300 as g

X = torch.rand(50, 8)
S = torch.eye(8, dtype=torch.float64)
PSI = torch.ones(8, dtype=torch.float64)

CALLS = {
    "preprocess": lambda: g.preprocess(X),
    "gram": lambda: g.gram(X),
    "spectra": lambda: g.spectra(S, 4),
    "lift": lambda: g.lift(X, S[:, :4].contiguous(), torch.ones(4, dtype=torch.float64), 4),
    "eigsolve": lambda: g.eigsolve([torch.ones(4, dtype=torch.float64), PSI]),
    "topk_network": lambda: g.topk_network(X, PSI, 3),
    "topk_network_gram": lambda: g.topk_network_gram(S, PSI, 3),
    "fit_two_axis": lambda: g.fit_two_axis(X, 4, 8, 3, 3),
}


@pytest.mark.parametrize("name", sorted(CALLS))
def test_cpu_input_raises(name):
    with pytest.raises((RuntimeError, ValueError, ImportError)):
        CALLS[name]()
