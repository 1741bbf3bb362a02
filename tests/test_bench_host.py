"""Host-side pieces of bench.py (no GPU): the roofline byte counts against
the workload table, and the density experiment's input generator."""
import numpy as np
import pytest

import workloads


def test_algorithmic_bytes_match_the_workload_table():
    import bench

    # one read of [A | b], one write of the r x (d+1) sketch, r row indices
    p2 = workloads.Problem(A=np.zeros((1 << 20, 64), np.float32), b=np.zeros(1 << 20, np.float32),
                           x_true=np.zeros(64), r=4096, seed=0)
    assert bench.algorithmic_bytes(p2, 4) == (1 << 20) * 65 * 4 + 4096 * 65 * 4 + 4 * 4096 == 273711104
    p1 = workloads.Problem(A=np.zeros((4096, 20)), b=np.zeros(4096), x_true=np.zeros(20), r=512, seed=0)
    assert bench.algorithmic_bytes(p1, 8) == 4096 * 21 * 8 + 512 * 21 * 8 + 4 * 512


@pytest.mark.parametrize("density", [0.02, 0.64])
def test_density_matrix_on_the_host(density):
    torch = pytest.importorskip("torch")
    import bench

    X = bench.density_matrix(20000, 11, density, seed=3, dev=torch.device("cpu")).numpy()
    assert X.shape == (20000, 11)
    frac = np.count_nonzero(X) / X.size
    assert abs(frac - density) < 4 * np.sqrt(density * (1 - density) / X.size) + 1e-3
    nz = X[X != 0]
    assert nz.min() > 0 and nz.max() <= 1.0
    # |N(0,1)| clipped at 1: about 68 % of the non-zeros are below 1, the rest equal 1
    assert abs(np.mean(nz < 1.0) - 0.6827) < 0.03
