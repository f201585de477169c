"""Pins for oracle.spectral, oracle.general, oracle.shybrid and oracle.rank."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import diffusion as D
from oracle import general, graph, rank, shybrid
from oracle import spectral as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return rows


def test_spectrum_facts(small_graph):
    # Sec. 3: eigenvalues in [-1, 1]; Sec. 4.4: lambda_1 = 1 and lambda_n <= -1/(n-1).
    W, A = small_graph["W"], small_graph["A"]
    lam, U = S.eigh_desc(W)
    n = lam.size
    assert lam[0] == pytest.approx(1.0, abs=1e-12)
    assert lam[-1] >= -1 - 1e-12 and lam[0] <= 1 + 1e-12
    assert lam[-1] <= -1.0 / (n - 1) + 1e-12
    ncomp, _ = S.components(A)
    assert np.sum(lam > 1 - 1e-9) == ncomp
    if ncomp == 1:
        sd = np.sqrt(np.asarray(A.sum(1)).ravel())
        u = U[:, 0] * np.sign(U[:, 0].sum())
        assert np.allclose(u, sd / np.linalg.norm(sd), atol=1e-10)


def test_multiplicity_equals_components():
    X1, _ = synth.database(21, 20, 4, 1, 40.0, 40.0)
    X2, _ = synth.database(22, 20, 4, 1, 40.0, 40.0)
    A = sp.block_diag([graph.adjacency(X1, 4), graph.adjacency(X2, 4)]).tocsr()
    W, _ = graph.normalize(A)
    lam, _ = S.eigh_desc(W)
    ncomp, _ = S.components(A)
    assert ncomp >= 2
    assert np.sum(lam > 1 - 1e-9) == ncomp


def test_orthogonality_eq5(small_graph):
    lam, U = S.eigh_desc(small_graph["W"])
    r = 7
    U1, U2 = U[:, :r], U[:, r:]
    assert np.allclose(U1.T @ U1, np.eye(r), atol=1e-12)
    assert np.allclose(U2.T @ U2, np.eye(60 - r), atol=1e-12)
    assert np.allclose(U1.T @ U2, 0, atol=1e-12)
    assert np.allclose(U1 @ U1.T + U2 @ U2.T, np.eye(60), atol=1e-12)


def test_theorem1_matrix_identity(small_graph):
    # Eq. 15: h(W) = U1 g(Lambda1) U1^T + h(W - U1 Lambda1 U1^T), dense, several r.
    W = small_graph["W"].toarray()
    hW = D.closed_form(W, np.eye(60), 0.99)
    for r in (0, 1, 6, 33, 60):
        lam, U = S.eigenpairs(W, r)
        rhs = (U * D.g_alpha(lam, 0.99)) @ U.T + D.closed_form(S.deflated(W, U, lam), np.eye(60), 0.99)
        assert np.allclose(hW, rhs, atol=1e-10)


def test_theorem2_polynomial(small_graph):
    # Appendix A, Eq. 32, for h(x) = 0.3 + 0.5x - 0.2x^2 + 0.1x^5.
    W = small_graph["W"]
    coeffs = [0.3, 0.5, -0.2, 0.0, 0.0, 0.1]
    y = np.random.default_rng(1).standard_normal(60)
    lam, U = S.eigenpairs(W, 9)
    direct = general.poly_apply(lambda z: W @ z, coeffs, y)
    assert np.allclose(general.hybrid_poly(W, U, lam, coeffs, y), direct, atol=1e-12)


def test_poly_apply_against_dense_spectral_evaluation(small_graph):
    # h(W) y for a polynomial h by Horner's rule equals V h(Lambda) V^T y from a
    # full dense eigendecomposition and the sum of explicit matrix powers.
    W = small_graph["W"].toarray()
    coeffs = [0.3, 0.5, -0.2, 0.0, 0.0, 0.1]
    y = np.random.default_rng(2).standard_normal(60)
    lam, V = np.linalg.eigh(W)
    ref = V @ (np.polyval(coeffs[::-1], lam) * (V.T @ y))
    powers = sum(c * (np.linalg.matrix_power(W, i) @ y) for i, c in enumerate(coeffs))
    got = general.poly_apply(lambda z: W @ z, coeffs, y)
    assert np.allclose(got, ref, atol=1e-12)
    assert np.allclose(got, powers, atol=1e-12)


def test_kappa_formulas(small_graph):
    # Eq. 22 and Eq. 23 against condition numbers of the dense matrices.
    W = small_graph["W"].toarray()
    lam, U = S.eigh_desc(W)
    a = 0.99
    L = (np.eye(60) - a * W) / (1 - a)
    assert S.kappa_of(L) == pytest.approx(S.kappa_laplacian(a, 1.0, lam[-1]), rel=1e-9)
    for r in (1, 3, 8):
        if lam[r] <= 0:
            continue
        Wr = S.deflated(W, U[:, :r], lam[:r])
        Lr = (np.eye(60) - a * Wr) / (1 - a)
        assert S.kappa_of(Lr) == pytest.approx(S.kappa_laplacian(a, lam[r], lam[-1]), rel=1e-9)


def test_worked_kappa_ratio_golden():
    # Sec. 4.4: alpha = 0.99, lambda_{r+1} = 0.7 gives the ratio 0.0326.
    (alpha, lam, ratio, digits), = _golden_rows("kappa_ratio.txt")
    got = S.kappa_laplacian(alpha, lam, -0.5) / S.kappa_laplacian(alpha, 1.0, -0.5)
    assert float(f"{got:.{int(digits)}g}") == ratio


def test_cg_error_within_bound(small_graph):
    # Eq. 21: ||e_i||_A / ||e_0||_A <= phi_i(A) at every iteration.
    W = small_graph["W"]
    a = 0.99
    y = np.zeros(60)
    y[[3, 17, 40]] = [1.0, 0.5, 0.25]
    for r in (0, 5):
        lam, U = S.eigenpairs(W, r)
        Wr = S.deflated(W, U, lam)
        Lr = (np.eye(60) - a * Wr) / (1 - a)
        xstar = np.linalg.solve(Lr, y)
        kap = S.kappa_of(Lr)
        errs = []
        D.cg(lambda z: Lr @ z, y, 1e-14, 200, callback=lambda i, x: errs.append(S.a_norm(Lr, xstar - x)))
        e0 = errs[0]
        for i, e in enumerate(errs):
            assert e / e0 <= S.phi(kap, i) + 1e-12


def test_table1_memory_golden():
    # Table 1: an n x r FP64 embedding of the 933,412-node component with r = 5k
    # takes 35,606 MB, i.e. MiB (2^20 bytes), truncated (35,606.5 exactly).
    (n, r, b, mb), = _golden_rows("table1_memory.txt")
    assert int(n * r * b // 2 ** 20) == mb


def test_sparsify_keeps_largest_magnitudes():
    U = np.array([[0.1, -0.5, 0.02], [0.3, -0.02, 0.9]])
    out = shybrid.sparsify(U, 0.5)
    assert np.count_nonzero(out) == 3
    assert set(np.abs(out[out != 0])) == {0.5, 0.3, 0.9}
    # equal magnitudes: the later (row-major) entry goes first
    out2 = shybrid.sparsify(U, 4 / 6)
    assert np.count_nonzero(out2) == 2 and out2[0, 1] == -0.5 and out2[1, 2] == 0.9
    out3 = shybrid.sparsify(np.array([[0.2, -0.2, 0.2]]), 1 / 3)
    assert list(out3[0]) == [0.2, -0.2, 0.0]


def test_topk_matches_python_sort():
    rng = np.random.default_rng(3)
    x = rng.integers(0, 6, 50).astype(float) / 7  # many ties
    for K in (1, 5, 50):
        ids, sc = rank.topk(x, K)
        want = sorted(range(50), key=lambda i: (-x[i], i))[:K]
        assert list(ids) == want
        assert np.array_equal(sc, x[want])


def test_pooled_and_rank_match():
    x = np.arange(12, dtype=float)
    assert list(rank.pooled(x, 3)) == [3, 12, 21, 30]
    ref = np.array([1.0, 1.0 + 1e-9, 0.5])
    assert rank.ranks_match([1, 0, 2], [0, 1, 2], ref, 1e-6)
    assert not rank.ranks_match([2, 0, 1], [0, 1, 2], ref, 1e-6)


def test_ranks_match_rejects_invalid_rankings():
    # Sec. 3: items ranked by decreasing score; a ranking may differ from the
    # reference only inside score ties, and must still be a ranking.
    ref = np.array([1.0, 1.0, 1.0, 0.5, 0.2])
    ids_ref, _ = rank.topk(ref, 3)
    assert list(ids_ref) == [0, 1, 2]
    assert rank.ranks_match([2, 0, 1], ids_ref, ref, 1e-9)            # a reordered tie run
    assert not rank.ranks_match([0, 0, 1], ids_ref, ref, 1e-9)        # an id twice inside the tie run
    assert not rank.ranks_match([0, 1, 5], ids_ref, ref, 1e-9)        # id out of range
    assert not rank.ranks_match([0, 1, 3], ids_ref, ref, 1e-9)        # 0.5 is not tied with 1.0
    assert not rank.ranks_match([0, 1], ids_ref, ref, 1e-9)           # wrong length
    # a ranking shifted down a chain of near-ties leaves out an item that belongs in it
    chain = np.array([5.0, 4.9, 4.8, 4.7, 0.0])
    cref, _ = rank.topk(chain, 3)
    assert rank.ranks_match([1, 0, 2], cref, chain, 0.15)
    assert not rank.ranks_match([1, 2, 3], cref, chain, 0.15)
    # the ranking's own scores: equal to the ranked vector at the ids, non-increasing,
    # equal scores with the smaller id first
    x = np.array([1.0, 1.0, 1.0, 0.5, 0.2], dtype=np.float32)
    assert rank.ranks_match([0, 1, 2], ids_ref, ref, 1e-9, scores=x[[0, 1, 2]], x=x)
    assert not rank.ranks_match([0, 1, 2], ids_ref, ref, 1e-9, scores=[1.0, 1.0, 0.9], x=x)
    assert not rank.ranks_match([1, 0, 2], ids_ref, ref, 1e-9, scores=x[[1, 0, 2]], x=x)
    y = np.array([1.0, 1.0 + 1e-12, 1.0, 0.5, 0.2])
    assert rank.ranks_match([1, 0, 2], ids_ref, ref, 1e-9, scores=y[[1, 0, 2]], x=y)
    assert not rank.ranks_match([0, 1, 2], ids_ref, ref, 1e-9, scores=y[[0, 1, 2]], x=y)
    # pooled scores: equal within a relative tolerance
    assert rank.ranks_match([0, 1, 2], ids_ref, ref, 1e-9, scores=[1.0 + 1e-8, 1.0, 1.0], x=ref,
                            score_tol=1e-6)


def test_kappa_deflated_against_dense(small_graph):
    # Sec. 4.4: W_r keeps r zero eigenvalues; for every r (including r with
    # lambda_{r+1} < 0, where Eq. 23 alone would not apply) the condition
    # number of the dense L_alpha(W_r) is the clamped formula.
    W = small_graph["W"].toarray()
    lam, U = S.eigh_desc(W)
    a = 0.99
    seen_negative = False
    for r in (0, 1, 4, 20, 45, 58):
        Wr = S.deflated(W, U[:, :r], lam[:r])
        Lr = (np.eye(60) - a * Wr) / (1 - a)
        lam_next = lam[r] if r > 0 else 1.0
        seen_negative |= lam_next < 0
        assert S.kappa_of(Lr) == pytest.approx(S.kappa_deflated(a, lam_next, lam[-1]), rel=1e-9)
    assert seen_negative


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-6])
def test_iteration_bound_holds_for_cg_and_pcg(small_graph, tol):
    # Eq. 21 turned into an iteration count: CG on the deflated operator (Form P)
    # and PCG with exact eigenpairs (Form S) never need more iterations than the
    # bound for the residual stopping rule, and the A-norm error is below tol
    # after iters_anorm iterations.
    W = small_graph["W"]
    Wd = W.toarray()
    a = 0.99
    lam, U = S.eigh_desc(Wd)
    Y = np.zeros((60, 3))
    Y[[3, 17, 40], 0] = [1.0, 0.5, 0.25]
    Y[[5, 6], 1] = [1.0, 1.0]
    Y[:, 2] = np.random.default_rng(4).random(60)
    L = (np.eye(60) - a * Wd) / (1 - a)
    kap_L = S.kappa_of(L)
    for r in (0, 3, 12):
        lam_next = lam[r] if r > 0 else 1.0
        kap = S.kappa_deflated(a, lam_next, lam[-1])
        Lr = (np.eye(60) - a * S.deflated(Wd, U[:, :r], lam[:r])) / (1 - a)
        i_res = S.cg_iterations_bound(kap, tol, kap)
        i_a = S.cg_iterations_bound(kap, tol)
        # minimality of both counts
        assert np.sqrt(kap) * S.phi(kap, i_res) <= tol < np.sqrt(kap) * S.phi(kap, i_res - 1) if i_res > 0 else True
        assert S.phi(kap, i_a) <= tol < (S.phi(kap, i_a - 1) if i_a > 0 else np.inf)
        for j in range(3):
            y = Y[:, j]
            xstar = np.linalg.solve(Lr, y)
            errs = []
            res = D.cg(lambda z: Lr @ z, y, tol, 500, callback=lambda i, x: errs.append(S.a_norm(Lr, xstar - x)))
            assert res.converged and res.iters <= i_res
            if len(errs) > i_a:
                assert errs[i_a] / errs[0] <= tol
            if r > 0:
                _, it = D.hybrid_pcg(W, U[:, :r], lam[:r], y, a, tol, 500)
                assert it[0] <= S.cg_iterations_bound(kap, tol, kap_L)
