"""Operation/byte accounting against the counts and tables the paper prints
(Sec. 3 text; Sec. 4, Tables 1 and 2).  Fixtures: tests/golden/paper_*.txt."""
import os

from paper_1411_2087_gb300 import metrics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _counts():
    out = {}
    with open(os.path.join(GOLDEN, "paper_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = int(v)
    return out


def _tables():
    rows = []
    with open(os.path.join(GOLDEN, "paper_tables.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                t, stream, soalen, ug, ub, cg, cb = line.split()
                rows.append((int(t), stream == "Yes", int(soalen), float(ug), float(ub),
                             float(cg), float(cb)))
    return rows


def test_dslash_counts_match_paper():
    c = _counts()
    assert metrics.matvec_flops() == c["matvec_real_multiplies"] + c["matvec_real_adds"]
    assert metrics.dslash_flops_per_site() == c["dslash_flops_per_site"]
    assert (c["dslash_matvecs_per_site"] * c["matvec_real_multiplies"]
            == c["dslash_real_multiplies_per_site"])
    # 16 matrices of 18 reals + 16 vectors of 6 reals
    assert (metrics.N_LINKS_NAIK * metrics.REALS_PER_LINK
            + metrics.N_LINKS_NAIK * metrics.REALS_PER_VECTOR) == c["dslash_input_operands_per_site"]


def test_multishift_models_match_paper():
    c = _counts()
    assert metrics.multishift_memory_bytes_per_site(9) == c["multishift_bytes_per_site_nm9"]
    assert metrics.multishift_memory_bytes_per_site(11) == c["multishift_bytes_per_site_nm11"]
    V = 1000
    assert metrics.multishift_cg_flops_per_iteration(V, 0) == c["cg_flops_per_site_base"] * V
    assert (metrics.multishift_cg_flops_per_iteration(V, 2)
            - metrics.multishift_cg_flops_per_iteration(V, 1)) == c["cg_flops_per_site_per_mass"] * V


def test_byte_model_reproduces_paper_tables():
    """GB/s = GF/s / flops_per_site * bytes_per_site with 4-byte reals, 16
    (Naik) or 8 (naive, 570 flops) links, 18 or 12 reals per link, and an extra
    output read without streaming stores: every printed GB/s within 1 GB/s."""
    for table, streaming, soalen, ug, ub, cgf, cgb in _tables():
        n_links = metrics.N_LINKS_NAIK if table == 2 else metrics.N_LINKS_NAIVE
        flops = metrics.dslash_flops_per_site(n_links)
        for gf, gb, rpl in ((ug, ub, metrics.REALS_PER_LINK),
                            (cgf, cgb, metrics.REALS_PER_LINK_COMPRESSED)):
            by = metrics.dslash_bytes_per_site(4, n_links, rpl, streaming)
            assert abs(gf / flops * by - gb) <= 1.0, (table, streaming, soalen, gf, gb)


def test_gpu_byte_model():
    assert metrics.dslash_bytes_per_site(8) == 2400
    assert metrics.dslash_bytes_per_site(4) == 1200
    assert metrics.dslash_half_bytes_per_site() == 608
    assert metrics.dslash_bytes_per_site(8, reals_per_link=12) == 1632
