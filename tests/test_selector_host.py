"""Host logic of the learned selector (no GPU): the class table, the paper's
decision tree restated on the library's features (Section 4.7), and the
regret measure the selector is judged by."""
import torch

from paper_2008_03909_gb300 import MLP_OUT
from paper_2008_03909_gb300 import selector as sel


def _feat(avg_deg, l_max_frac=0.9, depth=1.0):
    f = torch.zeros(16)
    f[2] = avg_deg
    f[11] = l_max_frac
    f[15] = depth
    return f


def test_class_table():
    # {k-out, BFS, LDD} x {UF-Rem-CAS, UF-Async, SV, LT-PRF}, in the order
    # the library's selected path numbers them (4 * sampling + finish)
    assert len(sel.CLASSES) == MLP_OUT == 12
    assert sel.CLASSES[sel.DEFAULT] == ("kout", "uf_rem_cas") and sel.DEFAULT == 0
    assert len(set(sel.CLASSES)) == len(sel.CLASSES)
    assert [s for s, _ in sel.CLASSES] == ["kout"] * 4 + ["bfs"] * 4 + ["ldd"] * 4
    assert [f for _, f in sel.CLASSES[:4]] == ["uf_rem_cas", "uf_async", "sv", "lt_prf"]
    so, fo = sel.class_opts(1)
    assert so.kind == 1 and fo.kind == 1 and fo.find == 1   # k-out, UF-Async with FindSplit


def test_paper_decision_tree_branches():
    # sparse graphs: no sampling; dense and shallow: BFS; otherwise k-out
    assert sel.paper_decision_tree(_feat(1.2)) == ("none", "uf_rem_cas")
    assert sel.paper_decision_tree(_feat(2.99, depth=0.0)) == ("none", "uf_rem_cas")
    assert sel.paper_decision_tree(_feat(16.0, depth=1.0)) == ("bfs", "uf_rem_cas")
    assert sel.paper_decision_tree(_feat(16.0, depth=4.0)) == ("kout", "uf_rem_cas")
    assert sel.paper_decision_tree(_feat(3.0, depth=5.0)) == ("kout", "uf_rem_cas")
    # shallow trees but no giant cluster: not a low-diameter graph
    assert sel.paper_decision_tree(_feat(16.0, l_max_frac=0.01, depth=1.0)) == ("kout", "uf_rem_cas")


def test_regret_definition():
    t = torch.tensor([[2.0, 1.0, 4.0], [3.0, 3.0, 6.0]])
    r = sel.regret(t, torch.tensor([0, 2]))
    assert torch.allclose(r, torch.tensor([1.0, 1.0]))
    r0 = sel.regret(t, torch.tensor([1, 0]))
    assert torch.allclose(r0, torch.zeros(2))
