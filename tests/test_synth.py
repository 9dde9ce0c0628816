"""The seeded workload recipe: ensemble members and joint weight clustering
(k-means) behave as their definitions state."""
import numpy as np

import synth


def test_kmeans_fixed_point_and_nearest_assignment():
    rng = np.random.default_rng(4)
    pts = rng.normal(size=(3000, 3))
    cent, assign = synth.kmeans(pts, 16)
    assert cent.shape == (16, 3) and assign.shape == (3000,)
    # every point sits with its nearest centroid (exact distances)
    d2 = ((pts[:, None, :] - cent[None, :, :]) ** 2).sum(axis=2)
    best = d2.min(axis=1)
    assert np.all(d2[np.arange(3000), assign] <= best + 1e-12)
    # every non-empty centroid is the mean of its points
    for j in range(16):
        sel = assign == j
        if sel.any():
            assert np.allclose(cent[j], pts[sel].mean(axis=0))


def test_kmeans_recovers_separated_clusters_and_is_deterministic():
    rng = np.random.default_rng(5)
    centres = np.array([[-10.0, 0.0], [0.0, 10.0], [10.0, 0.0]])
    pts = np.concatenate([c + 0.1 * rng.normal(size=(200, 2)) for c in centres])
    cent, assign = synth.kmeans(pts, 3)
    got = sorted(map(tuple, np.round(cent)))
    assert got == sorted(map(tuple, centres))
    cent2, assign2 = synth.kmeans(pts, 3)
    assert np.array_equal(cent, cent2) and np.array_equal(assign, assign2)


def test_k_at_least_distinct_points_is_exact():
    pts = np.array([[1.0], [2.0], [2.0], [5.0]])
    cent, assign = synth.kmeans(pts, 4)
    assert np.array_equal(cent[assign, 0], pts[:, 0])


def test_cluster_joint_shares_one_codebook_per_layer():
    net = synth.resnet18_mini()
    raws = [synth.params(net, m) for m in range(3)]
    cl = synth.cluster_joint(raws, net, 4)
    for i, nd in enumerate(net):
        if nd["op"] in ("conv", "dense"):
            # one centroid vector per position, at most 4 per layer
            vecs = np.stack([cl[m][i]["w"].reshape(-1) for m in range(3)], axis=1)
            assert len(np.unique(vecs, axis=0)) <= 4
        elif nd["op"] == "act":
            # the members share the activation polynomial
            assert cl[0][i] == cl[1][i] == cl[2][i]
    # members differ before clustering
    i = next(i for i, nd in enumerate(net) if nd["op"] == "conv")
    assert not np.array_equal(raws[0][i]["w"], raws[1][i]["w"])


def test_paper_parameter_sets_match_the_printed_chains():
    """synth's copy of the paper's ResNet-32 chain equals the appendix's
    printed chain (tests/golden/paper_primes.txt), q_0 first."""
    import paper_chains
    logn, d, q, p = paper_chains.chain("ResNet-32")
    pp = synth.PAPER_PARAMS["resnet32"]
    assert (pp["logn"], pp["log_scale"], pp["L"]) == (logn, d, len(q) - 1)
    assert pp["q"] == q and pp["p"] == p and pp["alpha"] == len(p)
