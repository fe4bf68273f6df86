"""Host pieces of the reconstruction driver: Poisson transmission noise
follows Beer-Lambert counting statistics (unbiased to first order, variance
1 / (I0 exp(-p)) of the log), and is reproducible from its seed."""
import numpy as np
import torch

from paper_2404_19075_b300.reconstruct import poisson_transmission


def test_poisson_transmission_statistics():
    p = torch.full((200000,), 0.7, dtype=torch.float64)
    i0 = 1e4
    y = poisson_transmission(p, i0, 5)
    mean_counts = i0 * np.exp(-0.7)
    assert abs(float(y.mean()) - 0.7) < 3e-3
    assert abs(float(y.var()) * mean_counts - 1.0) < 0.03
    assert torch.equal(y, poisson_transmission(p, i0, 5))
    assert not torch.equal(y, poisson_transmission(p, i0, 6))
    # no photons through: counts clamped to one, a finite line integral
    z = poisson_transmission(torch.full((10,), 50.0, dtype=torch.float64), 100.0, 1)
    assert torch.isfinite(z).all()
