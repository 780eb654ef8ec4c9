"""The input generator: the normal matrix it assembles block by block (and,
for the diffuse sky, summed per pointing position) equals the plain product
H^T W H of its own design matrix, and its workloads have the shapes the
method is exercised on."""
import numpy as np
import pytest

from spigen import SKY, TINY, generate, sky_scaled


@pytest.mark.parametrize("cfg", [TINY, sky_scaled(300, 4.0, 20), sky_scaled(400, 3.0, 10, seed=3)])
def test_normal_matrix_is_the_product_of_the_design(cfg):
    pb = generate(cfg, dense_design=True)
    H, w, y = pb.H, pb.w, pb.y
    N = H.T @ (H * w[:, None])
    A = pb.full_matrix().toarray()
    assert np.abs(A - N).max() <= 1e-13 * np.abs(N).max()
    assert np.array_equal(A != 0, N != 0)  # stored pattern = structural nonzeros
    b = H.T @ (w * y)
    assert np.abs(pb.b - b).max() <= 1e-13 * np.abs(b).max()


def test_sky_columns_and_full_rank():
    pb = generate(sky_scaled(300, 4.0, 20), dense_design=True)
    assert pb.n_sky > 0 and np.all(pb.kind[pb.sky_columns] == 3)
    assert np.all(np.abs(pb.H[:, pb.sky_columns]).sum(axis=0) > 0)  # every pixel seen
    ev = np.linalg.eigvalsh(pb.full_matrix().toarray())
    assert ev[0] > 0


def test_noise_free_sky_problem_has_x_true_as_solution():
    pb = generate(sky_scaled(300, 4.0, 20), noise=False)
    x = np.linalg.solve(pb.full_matrix().toarray(), pb.b)
    assert np.abs(x - pb.x_true).max() <= 1e-8 * np.abs(pb.x_true).max()


def test_sky_benchmark_member_shape():
    # the benchmark member: P = 8,000 on a 7 x 7 target grid, 1 deg pixels over 70 deg
    assert SKY.targets == 7 and SKY.sky_pix_deg == 1.0 and SKY.n_pointings == 8000
