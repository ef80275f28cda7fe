"""Seeded input generators: the von Mises-Fisher recipe of the deep-feature workload, on the host and
with torch (the device generator, run here on the CPU), against the closed form of the mean cosine
to the mean direction, E[w] = I_{d/2}(kappa) / I_{d/2-1}(kappa)."""
import numpy as np
import pytest

from paper_1705_01813_gb300 import datagen


def _mean_resultant(X):
    return float(np.linalg.norm(X.astype(np.float64).mean(0)))


def _a_d(kappa, d):
    special = pytest.importorskip("scipy.special")
    return float(special.ive(d / 2.0, kappa) / special.ive(d / 2.0 - 1.0, kappa))


@pytest.mark.parametrize("d,kappa", [(512, 50.0), (64, 20.0)])
def test_vmf_mean_cosine_host(d, kappa):
    # one direction: the mean of the samples is E[w] mu plus noise of norm ~ sqrt(1 / n)
    n = 20000
    X = datagen.bf16_bits_to_f32(datagen.deep_like(n, d, 1, kappa, seed=3))
    assert abs(_mean_resultant(X) - _a_d(kappa, d)) < 0.01 * _a_d(kappa, d) + 2.0 / n ** 0.5 / d ** 0.5


@pytest.mark.parametrize("d,kappa", [(512, 50.0), (64, 20.0)])
def test_vmf_mean_cosine_device_generator(d, kappa):
    torch = pytest.importorskip("torch")
    n = 20000
    X = datagen.deep_like_device(n, d, 1, kappa, seed=4, device="cpu", chunk=4096)
    assert X.dtype == torch.bfloat16 and X.shape == (n, d)
    Xf = X.float().numpy()
    assert abs(_mean_resultant(Xf) - _a_d(kappa, d)) < 0.01 * _a_d(kappa, d) + 2.0 / n ** 0.5 / d ** 0.5
    nrm = np.linalg.norm(Xf, axis=1)
    assert np.abs(nrm - 1.0).max() < 2e-3  # unit vectors up to BF16 rounding (2^-9 per element, relative)
    again = datagen.deep_like_device(n, d, 1, kappa, seed=4, device="cpu", chunk=4096)
    assert torch.equal(X, again)  # seeded


def test_vmf_mixture_host_and_device_agree():
    torch = pytest.importorskip("torch")
    n, d, dirs = 3000, 512, 200
    A = datagen.deep_like_device(n, d, dirs, 50.0, seed=7, device="cpu", chunk=1024).float()
    B = torch.from_numpy(datagen.bf16_bits_to_f32(datagen.deep_like(n, d, dirs, 50.0, seed=7)))

    def nn_cos(M):
        S = M @ M.T
        S.fill_diagonal_(-2.0)
        return float(S.max(1).values.mean())

    assert abs(nn_cos(A) - nn_cos(B)) < 0.03 * nn_cos(B)


@pytest.mark.parametrize("shape", [0.3, 1.0, 10.0, 40.0])
def test_gamma_device_moments(shape):
    """Gamma(a, 1) has mean a and variance a (the device Beta draws are ratios of these)."""
    torch = pytest.importorskip("torch")
    g = torch.Generator()
    g.manual_seed(int(shape * 100))
    x = datagen.gamma_device(torch.full((200_000,), shape), g).double()
    se = (shape / 200_000) ** 0.5
    assert abs(x.mean().item() - shape) < 5 * se
    assert abs(x.var().item() - shape) < 0.03 * shape + 5 * se


def test_gist_device_generator_matches_host_recipe():
    torch = pytest.importorskip("torch")
    A = datagen.gist_like_device(20000, 96, 50, seed=5, device="cpu", chunk=4096).numpy().astype(np.float64)
    B = datagen.gist_like(20000, 96, 50, seed=5).astype(np.float64)
    assert A.shape == B.shape and 0.0 <= A.min() and A.max() <= 1.0  # FP32 may round an extreme draw to 0 or 1
    # Beta(2, 8) latent means (mean 0.2); the spread mixes the latent and the per-sample Beta draws
    assert abs(A.mean() - B.mean()) < 0.01 and abs(A.std() - B.std()) < 0.01
    assert abs(A.mean() - 0.2) < 0.01
