"""FP64 oracle for the differentiable segmented-NCC loss (test infrastructure only).

The paper defines the forward quantities; this module adds their derivatives,
worked out by the chain rule (the paper gives none).

Forward, for a fixed segmentation S_1..S_K (rectangles) with raw values k_i:
  kbar = sum_i n_i k_i / n (Eq. 7), c_i = k_i - kbar, c(x) the rendered c_i,
  E_k = sum_i n_i c_i^2 (weighted energy, as in the segmented NCC oracle);
  rho_k(o) = sum_x c(x) (f(o+x) - fbar(o)) / sqrt(E_f(o) E_k)        (Eq. 9, 17, 18)
  rho_t(o) = sum_x t0(x) (f(o+x) - fbar(o)) / sqrt(E_f(o) E_t)        (Eq. 1)
  with t0 = t - tbar, E_t = sum t0^2, E_f(o) = sum_x (f(o+x) - fbar(o))^2;
  L = sum_o (rho_k(o) - rho_t(o))^2.
Gradients, with g = 2 (rho_k - rho_t):
  dL/dk_j = sum_o g [(S_j(o) - n_j fbar(o)) / sqrt(E_f E_k) - rho_k n_j c_j / E_k]
  dL/df(p) = sum_{o : p in window(o)} [ a(o) c(p-o) - b(o) t0(p-o) + h(o) (fbar(o) - f(p)) ]
  where a = g / sqrt(E_f E_k), b = g / sqrt(E_f E_t), h = g (rho_k - rho_t) / E_f.
Every window is assumed non-uniform (E_f > 0), which holds for the float
workloads used here.
"""
from __future__ import annotations

import numpy as np
from numpy.lib.stride_tricks import sliding_window_view


def render(rects, kvals, W: int, H: int) -> np.ndarray:
    img = np.zeros((H, W))
    for (x, y, w, h), k in zip(np.asarray(rects), np.asarray(kvals, np.float64)):
        img[y:y + h, x:x + w] = k
    return img


def forward(f, t, rects, kvals) -> dict:
    """rho_k, rho_t maps (V, U) and the loss L, all FP64."""
    f = np.asarray(f, np.float64)
    t = np.asarray(t, np.float64)
    H, W = t.shape
    n = W * H
    rects = np.asarray(rects)
    nk = rects[:, 2] * rects[:, 3]
    kv = np.asarray(kvals, np.float64)
    kbar = float(np.sum(nk * kv) / n)
    c = render(rects, kv - kbar, W, H)
    ek = float(np.sum(nk * (kv - kbar) ** 2))
    t0 = t - t.mean()
    et = float(np.sum(t0 * t0))
    win = sliding_window_view(f, (H, W))  # (V, U, H, W)
    fbar = win.mean(axis=(2, 3))
    dev = win - fbar[:, :, None, None]
    ef = np.einsum("vuhw,vuhw->vu", dev, dev)
    num_k = np.einsum("vuhw,hw->vu", dev, c)
    num_t = np.einsum("vuhw,hw->vu", dev, t0)
    rho_k = num_k / np.sqrt(ef * ek)
    rho_t = num_t / np.sqrt(ef * et)
    loss = float(np.sum((rho_k - rho_t) ** 2))
    return {"rho_k": rho_k, "rho_t": rho_t, "loss": loss, "c": c, "t0": t0, "ek": ek, "et": et, "ef": ef,
            "fbar": fbar, "kbar": kbar, "nk": nk, "win": win}


def gradients(f, t, rects, kvals) -> dict:
    """Analytic dL/dk (K,) and dL/df (N, M), FP64."""
    fw = forward(f, t, rects, kvals)
    f = np.asarray(f, np.float64)
    H, W = fw["c"].shape
    V, U = fw["rho_k"].shape
    g = 2.0 * (fw["rho_k"] - fw["rho_t"])
    a = g / np.sqrt(fw["ef"] * fw["ek"])
    b = g / np.sqrt(fw["ef"] * fw["et"])
    h = g * (fw["rho_k"] - fw["rho_t"]) / fw["ef"]
    rects = np.asarray(rects)
    kv = np.asarray(kvals, np.float64)
    cvals = kv - fw["kbar"]
    # dL/dk_j: Gt(x) = sum_o a(o) f(o + x) summed over segment j
    gt = np.einsum("vuhw,vu->hw", fw["win"], a)
    a1 = float(np.sum(a * fw["fbar"]))
    a2 = float(np.sum(g * fw["rho_k"]))
    dk = np.empty(len(kv))
    for j, (x, y, w, hh) in enumerate(rects):
        nj = w * hh
        dk[j] = gt[y:y + hh, x:x + w].sum() - nj * a1 - nj * cvals[j] * a2 / fw["ek"]
    # dL/df: scatter every template position's contribution onto the window
    df = np.zeros_like(f)
    hf = h * fw["fbar"]
    for y in range(H):
        for x in range(W):
            df[y:y + V, x:x + U] += a * fw["c"][y, x] - b * fw["t0"][y, x] + hf - h * f[y:y + V, x:x + U]
    return {"dk": dk, "df": df, "loss": fw["loss"]}
