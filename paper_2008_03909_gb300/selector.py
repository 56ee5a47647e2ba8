"""Learned variant selector: picks ConnectIt's sampling x finish combination
for a graph from cheap features, with an MLP trained on the GPU by the
library's own kernels (cc_mlp_*).  It never changes labels: every class
runs the same exact connectivity, only faster or slower; if anything goes
wrong it falls back to k-out + UF-Rem-CAS.

Classes: {k-out (k = 2), BFS (3 tries), LDD (beta 0.2)} x {UF-Rem-CAS,
UF-Async, SV, Liu-Tarjan PRF}, class 0 (k-out + UF-Rem-CAS) the default.
The choice is made inside the selected path (cc_select_static): the
default's k-out sample is computed first, the features come from it, and a
k-out class continues on it, so the features cost little and the sample is
not redone.

The paper chooses by a hand-made decision tree (Section 4.7): UF-Rem-CAS
with FindNaive; no sampling when m/n < 3; BFS (or LDD) sampling for dense,
low-diameter graphs; k-out otherwise.  `paper_decision_tree` restates it on
this library's features; its no-sampling branch lies outside the twelve
classes, so it returns (sampling, finish) names rather than a class index.
"""
from __future__ import annotations

import torch

from . import (MLP_IN, MLP_NPARAM, MLP_OUT, cc_features, cc_select_static, cc_static, finish_opt, mlp_adam,
               mlp_backward, mlp_forward, mlp_init, mlp_predict, mlp_set_norm, mlp_soft_targets, sample_opt)

SAMPLES = ("kout", "bfs", "ldd")
FINISHES = ("uf_rem_cas", "uf_async", "sv", "lt_prf")
CLASSES = [(s, f) for s in SAMPLES for f in FINISHES]
assert len(CLASSES) == MLP_OUT
DEFAULT = CLASSES.index(("kout", "uf_rem_cas"))
assert DEFAULT == 0


def class_opts(c: int):
    """cc_static options of class c (the same combination cc_select_static
    runs for c)."""
    s, f = CLASSES[c]
    return sample_opt(s), finish_opt(f, "split" if f == "uf_async" else "naive")


def paper_decision_tree(feat: torch.Tensor) -> tuple:
    """The paper's rule on one feature vector (host floats): (sampling,
    finish).  Dense means m/n >= 3; low diameter means the k-out trees were
    shallow (at most 1.5 parent steps per non-root in the sampling's last
    compression) and the frequent cluster holds at least half the vertices."""
    f = [float(x) for x in feat]
    avg_deg, l_max_frac, depth = f[2], f[11], f[15]
    if avg_deg < 3.0:
        return ("none", "uf_rem_cas")
    if depth <= 1.5 and l_max_frac >= 0.5:
        return ("bfs", "uf_rem_cas")
    return ("kout", "uf_rem_cas")


def _timed(fn, reps: int) -> float:
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    best = float("inf")
    for _ in range(reps):
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def time_classes(offsets, edges, reps: int = 3, labels=None, realized: bool = True) -> torch.Tensor:
    """Milliseconds of every class on one graph (best of `reps` after one
    untimed run), with CUDA events on the current stream.  realized: each
    class as the selected path runs it (cc_select_static with the class
    forced: features and the default's k-out sample included, the sample
    reused by k-out classes); else as a plain cc_static call."""
    n = offsets.numel() - 1
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device=offsets.device)
    out = torch.empty(MLP_OUT, dtype=torch.float32)
    for c in range(MLP_OUT):
        if realized:
            out[c] = _timed(lambda: cc_select_static(offsets, edges, None, c, labels_out=labels), reps)
        else:
            so, fo = class_opts(c)
            out[c] = _timed(lambda: cc_static(offsets, edges, so, fo, labels), reps)
    return out


class Selector:
    """MLP 16 -> 64 -> 64 -> 12 over the selected path's features, trained
    on measured times."""

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
        """Labels of the graph by the selected path (features, choice and run
        in one call), and the class it ran; k-out + UF-Rem-CAS if the
        selected path cannot run."""
        try:
            return cc_select_static(offsets, edges, self.params, -1, labels_out=labels_out)
        except Exception:
            so, fo = class_opts(DEFAULT)
            return cc_static(offsets, edges, so, fo, labels_out), DEFAULT


def regret(times: torch.Tensor, choice: torch.Tensor) -> torch.Tensor:
    """(t_choice - t_best) / t_best per graph."""
    t = times.cpu()
    ch = choice.cpu().long()
    best = t.min(dim=1).values
    return t.gather(1, ch[:, None])[:, 0] / best - 1.0
