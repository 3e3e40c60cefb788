"""The seeded generators: SPD by construction and in the packed batch layout
(host NumPy recipes and their device-side counterparts, run here on the CPU)."""
import numpy as np
import pytest

import gen


def _min_eig(orc, D, E, G, R):
    return np.linalg.eigvalsh(orc.assemble_dense(D, E, G, R)).min()


def test_psd_couplings_keep_small_blocks_spd(orc):
    """n = 12 without an arrow: the embedded couplings give an SPD matrix
    for every draw (the plain couplings need not)."""
    for seed in range(20):
        D, E, G, R = gen.ipm(60, 12, 0, seed=seed, sigma_decades=6.0, psd_couplings=True)
        assert _min_eig(orc, D, E, G, R) > 0


@pytest.mark.parametrize("kind", ["ipm", "raceline"])
def test_device_batch_layout_and_spd(orc, kind):
    torch = pytest.importorskip("torch")
    import gen.device as gd
    Ns, ns, ms = [7, 12, 5], [3, 6, 3], [2, 0, 1]
    D, E, G, R = gd.batch(Ns, ns, ms, seed=3, kind=kind, psd_couplings=True, device="cpu")
    off = gd.offsets(Ns, ns, ms)
    assert D.numel() == off["D"][-1] and E.numel() == off["E"][-1]
    for s, (N, n, m) in enumerate(zip(Ns, ns, ms)):
        Ds = D[off["D"][s]:off["D"][s + 1]].reshape(N, n, n).numpy()
        Es = E[off["E"][s]:off["E"][s + 1]].reshape(N - 1, n, n).numpy()
        Gs = G[off["G"][s]:off["G"][s + 1]].reshape(N, m, n).numpy() if m else np.zeros((N, 0, n))
        Rs = R[off["R"][s]:off["R"][s + 1]].reshape(m, m).numpy() if m else np.zeros((0, 0))
        np.testing.assert_allclose(Ds, np.swapaxes(Ds, 1, 2), rtol=1e-12, atol=1e-9)
        assert _min_eig(orc, Ds, Es, Gs, Rs) > 0
