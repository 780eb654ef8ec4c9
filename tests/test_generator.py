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


@pytest.mark.parametrize("cfg", [TINY, sky_scaled(300, 4.0, 20)])
def test_oracle_normal_equations_match_the_generator(cfg):
    """The oracle's N = H^T W H, b = H^T W y (one sparse product of the
    design matrix) equals the generator's windowed / per-position assembly."""
    import oracle
    pb = generate(cfg, sparse_design=True)
    v, b = oracle.normal_equations(pb.H, pb.w, pb.y, pb.colptr, pb.rowind)
    assert np.abs(v - pb.values).max() <= 1e-13 * np.abs(pb.values).max()
    assert np.abs(b - pb.b).max() <= 1e-13 * np.abs(pb.b).max()


def test_oracle_normal_equations_closed_forms():
    """Diagonal H: N = diag(w h^2); a pattern entry with no product term is 0."""
    import oracle
    import scipy.sparse as sp
    h = np.array([2.0, -1.0, 0.5]); w = np.array([1.0, 3.0, 4.0]); y = np.array([1.0, 2.0, 3.0])
    H = sp.csr_matrix(np.diag(h))
    colptr = np.array([0, 2, 3, 4], np.int64); rowind = np.array([0, 2, 1, 2], np.int32)
    v, b = oracle.normal_equations(H, w, y, colptr, rowind)
    assert np.array_equal(v, [w[0] * h[0] ** 2, 0.0, w[1] * h[1] ** 2, w[2] * h[2] ** 2])
    assert np.array_equal(b, w * y * h)
