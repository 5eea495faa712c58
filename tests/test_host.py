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
