"""Learned variant selector: picks ConnectIt's sampling x finish combination
for a graph from cheap features, with an MLP trained on the GPU by the
library's own kernels (cc_mlp_*).  It never changes labels: every class
runs the same exact connectivity, only faster or slower; if anything goes
wrong it falls back to k-out + UF-Rem-CAS.

The paper chooses by a hand-made decision tree (Section 4.7):
UF-Rem-CAS with FindNaive; no sampling when m/n < 3; BFS (or LDD) sampling
for dense, low-diameter graphs; k-out otherwise.  `paper_decision_tree`
restates it on this library's features (low diameter: a BFS from the
highest-degree vertex finishes within 64 levels and reaches at least half
of the vertices).
"""
from __future__ import annotations

import torch

from . import (MLP_IN, MLP_NPARAM, MLP_OUT, cc_features, cc_static, finish_opt, mlp_adam, mlp_backward,
               mlp_forward, mlp_init, mlp_predict, mlp_set_norm, mlp_soft_targets, sample_opt)

SAMPLES = ("none", "kout", "bfs", "ldd")
FINISHES = ("uf_rem_cas", "uf_async", "sv")
CLASSES = [(s, f) for s in SAMPLES for f in FINISHES]
assert len(CLASSES) == MLP_OUT
DEFAULT = CLASSES.index(("kout", "uf_rem_cas"))


def class_opts(c: int):
    s, f = CLASSES[c]
    return sample_opt(s), finish_opt(f, "split" if f == "uf_async" else "naive")


def paper_decision_tree(feat: torch.Tensor) -> int:
    """The paper's rule on one feature vector (host floats)."""
    f = [float(x) for x in feat]
    avg_deg, bfs_levels, bfs_reached = f[2], f[14], f[15]
    if avg_deg < 3.0:
        return CLASSES.index(("none", "uf_rem_cas"))
    # low diameter: the capped BFS finished AND it covered most of the graph
    # (a hub inside a small component finishes early on any graph)
    if bfs_levels < 1.0 and bfs_reached >= 0.5:
        return CLASSES.index(("bfs", "uf_rem_cas"))
    return DEFAULT


def time_classes(offsets, edges, reps: int = 3, labels=None) -> torch.Tensor:
    """Milliseconds of every class on one graph (best of `reps` after one
    untimed run), with CUDA events on the current stream."""
    n = offsets.numel() - 1
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device=offsets.device)
    out = torch.empty(MLP_OUT, dtype=torch.float32)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for c in range(MLP_OUT):
        so, fo = class_opts(c)
        cc_static(offsets, edges, so, fo, labels)
        best = float("inf")
        for _ in range(reps):
            e0.record()
            cc_static(offsets, edges, so, fo, labels)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[c] = best
    return out


class Selector:
    """MLP 16 -> 64 -> 64 -> 12 over cc_features, trained on measured times."""

    def __init__(self, device="cuda", seed: int = 1):
        self.device = torch.device(device)
        self.params = torch.empty(MLP_NPARAM, dtype=torch.float32, device=self.device)
        mlp_init(self.params, seed)

    def fit(self, X: torch.Tensor, T: torch.Tensor, epochs: int = 400, lr: float = 3e-3, tau: float = 0.05):
        """X: float32[N,16] features, T: float32[N,12] milliseconds (CUDA).
        Full-batch Adam on the cross-entropy to soft targets exp(-regret/tau).
        Returns the loss history (host floats)."""
        X = X.to(self.device, torch.float32).contiguous()
        T = T.to(self.device, torch.float32).contiguous()
        B = X.shape[0]
        mlp_set_norm(self.params, X)
        Q = torch.empty(B, MLP_OUT, dtype=torch.float32, device=self.device)
        mlp_soft_targets(T, tau, Q)
        logits = torch.empty(B, MLP_OUT, dtype=torch.float32, device=self.device)
        acts = torch.empty(B, 128, dtype=torch.float32, device=self.device)
        grads = torch.zeros(MLP_NPARAM, dtype=torch.float32, device=self.device)
        m = torch.zeros_like(grads)
        v = torch.zeros_like(grads)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        hist = torch.empty(epochs, dtype=torch.float32, device=self.device)
        for step in range(1, epochs + 1):
            mlp_forward(self.params, X, logits, acts)
            mlp_backward(self.params, X, acts, logits, Q, grads, loss)
            hist[step - 1] = loss[0]
            mlp_adam(self.params, grads, m, v, step, lr)
        return hist.cpu().tolist()

    def predict(self, X: torch.Tensor) -> torch.Tensor:
        X = X.to(self.device, torch.float32).contiguous().reshape(-1, MLP_IN)
        out = torch.empty(X.shape[0], dtype=torch.int32, device=self.device)
        mlp_predict(self.params, X, out)
        return out

    def choose(self, offsets, edges) -> int:
        try:
            return int(self.predict(cc_features(offsets, edges)).item())
        except Exception:
            return DEFAULT

    def run(self, offsets, edges, labels_out=None):
        """Labels of the graph with the chosen combination (k-out + UF-Rem-CAS
        if the choice cannot run)."""
        c = self.choose(offsets, edges)
        so, fo = class_opts(c)
        try:
            return cc_static(offsets, edges, so, fo, labels_out), c
        except Exception:
            so, fo = class_opts(DEFAULT)
            return cc_static(offsets, edges, so, fo, labels_out), DEFAULT


def regret(times: torch.Tensor, choice: torch.Tensor) -> torch.Tensor:
    """(t_choice - t_best) / t_best per graph."""
    t = times.cpu()
    ch = choice.cpu().long()
    best = t.min(dim=1).values
    return t.gather(1, ch[:, None])[:, 0] / best - 1.0
