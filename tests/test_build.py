"""__graft_entry__.build() compiles the CUDA library (sm_103a) and the oracle."""
import os


def test_entry_build():
    import __graft_entry__ as g
    g.build()
    import paper_1606_09481_gb300 as rhg
    assert os.path.exists(rhg.LIB)
