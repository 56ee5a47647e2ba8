"""Host logic of the learned selector (no GPU): the class table, the paper's
decision tree restated on the library's features (Section 4.7), and the
regret measure the selector is judged by."""
import torch

from paper_2008_03909_gb300 import MLP_OUT
from paper_2008_03909_gb300 import selector as sel


def _feat(avg_deg, bfs_levels, reached=1.0):
    f = torch.zeros(16)
    f[2] = avg_deg
    f[14] = bfs_levels
    f[15] = reached
    return f


def test_class_table():
    assert len(sel.CLASSES) == MLP_OUT == 12
    assert sel.CLASSES[sel.DEFAULT] == ("kout", "uf_rem_cas")
    assert len(set(sel.CLASSES)) == len(sel.CLASSES)


def test_paper_decision_tree_branches():
    # sparse graphs: no sampling; dense low-diameter: BFS; otherwise k-out
    assert sel.CLASSES[sel.paper_decision_tree(_feat(1.2, 0.0))] == ("none", "uf_rem_cas")
    assert sel.CLASSES[sel.paper_decision_tree(_feat(2.99, 1.0))] == ("none", "uf_rem_cas")
    assert sel.CLASSES[sel.paper_decision_tree(_feat(16.0, 0.0))] == ("bfs", "uf_rem_cas")
    assert sel.CLASSES[sel.paper_decision_tree(_feat(16.0, 1.0))] == ("kout", "uf_rem_cas")
    assert sel.CLASSES[sel.paper_decision_tree(_feat(3.0, 5.0))] == ("kout", "uf_rem_cas")
    # the BFS finished early but inside a small component: not low diameter
    assert sel.CLASSES[sel.paper_decision_tree(_feat(16.0, 0.2, 0.01))] == ("kout", "uf_rem_cas")
    assert sel.CLASSES[sel.paper_decision_tree(_feat(16.0, 0.2, 0.5))] == ("bfs", "uf_rem_cas")


def test_regret_definition():
    t = torch.tensor([[2.0, 1.0, 4.0], [3.0, 3.0, 6.0]])
    r = sel.regret(t, torch.tensor([0, 2]))
    assert torch.allclose(r, torch.tensor([1.0, 1.0]))
    r0 = sel.regret(t, torch.tensor([1, 0]))
    assert torch.allclose(r0, torch.zeros(2))
