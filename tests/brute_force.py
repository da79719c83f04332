"""Brute-force all-pairs blender used to pin the oracle's tiled path.

Written independently of the oracle: for every pixel it scans ALL Gaussians,
keeps those whose tile rectangle contains the pixel's tile, orders them by
(float32 depth bits, index) and blends front to back with the early-stop rule
(alpha clamp 0.99, skip below 1/255, stop before transmittance < 1e-4).
Plain Python loops: only for tiny inputs (<= a few dozen Gaussians, <= 64x64).
"""
import math

import numpy as np


def blend_all_pairs(proj, w_ds, h_ds, d, ox, oy, tile, bg=(0.0, 0.0, 0.0)):
    n = proj["xy"].shape[0]
    dbits = np.asarray(proj["depth"], np.float64).astype(np.float32).view(np.uint32)
    img = np.zeros((h_ds, w_ds, 3))
    t_final = np.ones((h_ds, w_ds))
    for v in range(h_ds):
        for u in range(w_ds):
            tx, ty = u // tile, v // tile
            cand = []
            for g in range(n):
                x0, y0, x1, y1 = proj["rect"][g]
                if proj["tiles_touched"][g] > 0 and x0 <= tx <= x1 and y0 <= ty <= y1:
                    cand.append((int(dbits[g]), g))
            cand.sort()
            x, y = d * u + ox, d * v + oy
            T = 1.0
            C = [0.0, 0.0, 0.0]
            for _, g in cand:
                px, py = proj["xy"][g]
                A, B, Cc = proj["conic"][g]
                dx, dy = x - px, y - py
                power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy
                if power > 0:
                    continue
                alpha = min(0.99, proj["opacity"][g] * math.exp(power))
                if alpha < 1.0 / 255.0:
                    continue
                if T * (1 - alpha) < 1e-4:
                    break
                for ch in range(3):
                    C[ch] += proj["rgb"][g][ch] * alpha * T
                T *= 1 - alpha
            img[v, u] = [C[ch] + T * bg[ch] for ch in range(3)]
            t_final[v, u] = T
    return img, t_final
