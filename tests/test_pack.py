"""CPU checks of pack_instances, the argument builder of the packed batch
call: its arrays are the block-diagonal matrices scipy builds from the same
instances, and the instances' vectors concatenated."""
import numpy as np
import scipy.sparse as sp

import qpgen
from paper_2311_07710_gb300 import pdqp


def _bag():
    return [qpgen.tiny_qp(7 + k, n=3 + 4 * k, m=2 + 3 * k, m_eq=k, bounds="mixed", density=0.6) for k in range(4)] \
        + [qpgen.diagonal_box_qp(5, 9), qpgen.tiny_qp(30, n=6, m=0, m_eq=0)]


def test_pack_matches_block_diag():
    insts = _bag()
    p = pdqp.pack_instances(insts)
    assert list(p["n"]) == [i.n for i in insts] and list(p["m"]) == [i.m for i in insts]
    assert list(p["m_eq"]) == [i.m_eq for i in insts]
    N, M = sum(i.n for i in insts), sum(i.m for i in insts)
    for name, mats, rows in (("Q", [i.Q for i in insts], N), ("A", [i.A for i in insts], M)):
        ref = sp.csr_matrix(sp.block_diag(mats, format="csr"))
        ref.sort_indices()
        got = sp.csr_matrix((p[f"{name}_val"], p[f"{name}_col"], p[f"{name}_rowptr"]), shape=(rows, N))
        assert p[f"{name}_rowptr"].dtype == np.int32 and p[f"{name}_col"].dtype == np.int32
        assert len(p[f"{name}_rowptr"]) == rows + 1
        # same entries in the same positions (the instances' own order within a row)
        np.testing.assert_array_equal(got.indptr, ref.indptr)
        np.testing.assert_array_equal(got.indices, ref.indices)
        np.testing.assert_array_equal(got.data, ref.data)
    for f in ("c", "l", "u"):
        np.testing.assert_array_equal(p[f], np.concatenate([getattr(i, f) for i in insts]))
    np.testing.assert_array_equal(p["b"], np.concatenate([i.b for i in insts]))


def test_pack_columns_stay_inside_their_instance():
    insts = _bag()
    p = pdqp.pack_instances(insts)
    xoff = np.concatenate([[0], np.cumsum(p["n"])])
    yoff = np.concatenate([[0], np.cumsum(p["m"])])
    for k in range(len(insts)):
        for name, off in (("Q", xoff), ("A", yoff)):
            rp = p[f"{name}_rowptr"]
            cols = p[f"{name}_col"][rp[off[k]]:rp[off[k + 1]]]
            assert np.all((cols >= xoff[k]) & (cols < xoff[k + 1]))
