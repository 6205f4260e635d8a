"""Restoration-quality side report: signal-to-noise ratios of the blurred
image and of Wiener, RL, RRRL and WR3L restorations on synthetic test
images, the columns of the paper's SNR table (Sec. 3.1) that
this library implements (the comparison methods WYYZ and KF are not part of
it).  The paper's test images are not available; seeded synthetic scenes
stand in for them.

    SNR(u, u0) = 10 log10( var(u) / var(u - u0) ) dB

with u the blurred or restored image and u0 the sharp one (Sec. 3.1, as
printed).  Every restoration runs through the library on the GPU.

    python -m paper_1212_2245_b300.quality            # markdown table
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import deblur, rrl_iterate, synth, wiener
from .params import Params


def snr_db(u: torch.Tensor | np.ndarray, u0: torch.Tensor | np.ndarray) -> float:
    u = torch.as_tensor(u, dtype=torch.float64).cpu()
    u0 = torch.as_tensor(u0, dtype=torch.float64).cpu()
    return 10.0 * math.log10(float(u.var(unbiased=False) / (u - u0).var(unbiased=False)))


@dataclasses.dataclass
class QualityCase:
    name: str
    g: np.ndarray   # sharp image
    f: np.ndarray   # blurred, noisy image
    h: np.ndarray   # PSF
    kind: str       # "general" or "box"
    params: Params


def default_cases() -> list[QualityCase]:
    """Synthetic stand-ins: 256^2 scenes with horizontal box motion (lengths
    15 and 27, the latter the paper's length), a 30-degree line blur with
    salt-and-pepper noise and a Gaussian-mixture blur."""
    out = []
    specs = [
        ("box15 256^2, sigma 2", synth.box_psf(15), "box", 2.0, 0.0),
        ("box27 256^2, sigma 2", synth.box_psf(27), "box", 2.0, 0.0),
        ("box26.5 256^2, sigma 2", synth.box_psf_frac(26.5), "box", 2.0, 0.0),
        ("line31@30deg 256^2, sigma 2 + 1% s&p", synth.line_psf(31, 30.0, 32.0), "general", 2.0, 0.01),
        ("gauss15 256^2, sigma 1", None, "general", 1.0, 0.0),
    ]
    for k, (name, h, kind, sigma, sp) in enumerate(specs):
        rng = np.random.default_rng(20250 + k)
        if h is None:
            h = synth.gaussian_mixture_psf(15, rng)
        g = synth.scene(256, 256, rng).astype(np.float32)
        f = synth.degrade(g, h, sigma, rng, salt_pepper=sp)
        out.append(QualityCase(name, g, f, h.astype(np.float32), kind, Params()))
    return out


def _cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32).cuda()


def evaluate(case: QualityCase) -> dict[str, float]:
    """SNR of every column for one case."""
    f, h, p = _cuda(case.f), _cuda(case.h), case.params
    start = torch.clamp(f, min=p.pos_floor)  # RL and RRRL start from the observed image
    rl = dataclasses.replace(p, phi_robust=0, alpha=0.0)
    row = {"blurred": snr_db(case.f, case.g),
           f"Wiener (K={p.K})": snr_db(wiener(f, h, p, kind=case.kind), case.g),
           "RL 30 it.": snr_db(rrl_iterate(f, start.clone(), h, rl, 30, kind=case.kind), case.g)}
    for n in (5, 30, 100):
        row[f"RRRL {n} it."] = snr_db(rrl_iterate(f, start.clone(), h, p, n, kind=case.kind), case.g)
    row["WR3L 5 it."] = snr_db(deblur(f, h, p, 5, kind=case.kind), case.g)
    return row


def table(cases: list[QualityCase] | None = None) -> str:
    cases = cases if cases is not None else default_cases()
    rows = [(c.name, evaluate(c)) for c in cases]
    cols = list(rows[0][1].keys())
    lines = ["| test image | " + " | ".join(cols) + " |", "|---" * (len(cols) + 1) + "|"]
    for name, r in rows:
        lines.append(f"| {name} | " + " | ".join(f"{r[c]:.2f}" for c in cols) + " |")
    return "\n".join(lines)


if __name__ == "__main__":
    print(table())
