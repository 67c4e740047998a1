"""Oracle states along a horizon, for error-versus-step curves (test helper)."""
import dataclasses

import numpy as np

from paper_2503_22767_gb300 import workloads as W


def oracle_states(w, horizons, threads=None):
    """FP64 oracle states (x, v, C, F) after each substep count in
    ``horizons``.  The horizon runs in windows, each continuing from the
    previous window's double-precision state with the field (and box motion,
    field gradient) of its own substeps, so every state equals that of one
    straight run.  ``threads``: host threads (default all cores)."""
    import oracle

    cfg = w.cfg
    x = w.x0.astype(np.float64)
    v = np.zeros_like(x) if w.v0 is None else w.v0.astype(np.float64)
    C = F = None
    out, prev = {}, 0
    with oracle.threads(threads):
        for h in sorted(horizons):
            c = dataclasses.replace(cfg, n_steps=h - prev)
            seg = W.Workload(w.name, c, x, v, w.phi, w.mag, np.ascontiguousarray(w.field[:, prev:h]),
                             w.target, dict(w.meta),
                             None if w.bmotion is None else np.ascontiguousarray(w.bmotion[:, prev:h]),
                             None if w.fgrad is None else np.ascontiguousarray(w.fgrad[:, prev:h]))
            o = oracle.forward(seg, C0=C, F0=F)
            x, v, C, F = o["x"], o["v"], o["C"], o["F"]
            out[h] = dict(x=x, v=v, C=C, F=F)
            prev = h
    return out
