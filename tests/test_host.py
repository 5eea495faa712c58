"""Host-side logic of the learned proposal (no GPU)."""



def test_proposal_labels_and_parameter_layout():
    from paper_2502_11017_gb300 import proposal as prop
    import paper_2502_11017_gb300 as cur
    fam = dict(m=6, n=4)
    yr, yc = prop.labels([[0, 5], [2, 3]], [[1, 2], [0, 3]], family=fam)
    assert yr.tolist() == [1, 0, 0, 0, 0, 1, 0, 0, 1, 1, 0, 0]
    assert yc.tolist() == [0, 1, 1, 0, 1, 0, 0, 1]
    p = prop.init_params(0)
    assert p.size == cur.mlp_param_count(32, 256) == 32 * 256 + 2 * 256 + 1
    assert (p[32 * 256:32 * 256 + 256] == 0).all() and p[-1] == 0


def test_stored_proposal_labels_are_the_oracles_crosses():
    """tests/golden/proposal_labels_4096x1024_r16.npz holds what make_proposal_labels.py
    writes: re-derive three of its crosses with the oracle."""
    import os

    import numpy as np

    from oracle import cur_oracle as orc
    from paper_2502_11017_gb300 import workloads as wl
    path = os.path.join(os.path.dirname(__file__), "golden", "proposal_labels_4096x1024_r16.npz")
    lab = np.load(path)
    F = wl.PROPOSAL_FAMILY
    fam = wl.proposal_family(len(lab["seed"]), h_range=F["h_range"])
    assert [s for s, _ in fam] == lab["seed"].tolist()
    for t in (0, 1000, len(fam) - 1):
        seed, h = fam[t]
        assert h == lab["h"][t]
        a = wl.gaussian_kernel(F["m"], F["n"], h, seed=seed)
        I, J, info = orc.cross(a, F["r"], F["b_r"], F["b_c"])
        assert I == lab["I"][t].tolist() and J == lab["J"][t].tolist()
        assert info["logvol"] == lab["logvol"][t]
