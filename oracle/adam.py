"""Adam over the raw parameter planes, FP64 -- TEST INFRASTRUCTURE ONLY (the oracle of the
fused optimiser step; nothing on the product path imports it).

Adam (Kingma & Ba, "Adam: A Method for Stochastic Optimization", 2015, Algorithm 1), per
entry, with the bias corrections written as divisions:
    m <- b1 m + (1 - b1) g ;  v <- b2 v + (1 - b2) g^2
    x <- x - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
The optimised planes are raw: scale holds log s and opacity holds logit o (the 3D-GS
activations); the gradient given is w.r.t. the activated parameter, so g = g_act * act'(x).
Groups (learning rate, step): mean, scale, rot, opacity, SH band 0, SH bands >= 1, lobes.
A group with lr 0 is left untouched (the staged lobe introduction of Sec. "Implementation").
"""
import numpy as np

GROUPS = ("MEAN", "SCALE", "ROT", "OPACITY", "SH_DC", "SH_REST", "SG")
PLANES = ("mean", "scale", "rot", "opacity", "sh", "sg_amp", "sg_axis", "sg_sharp")


def activation(plane):
    return {"scale": "exp", "opacity": "sigmoid"}.get(plane, "identity")


def activate(kind, x):
    if kind == "exp":
        return np.exp(x)
    if kind == "sigmoid":
        return 1.0 / (1.0 + np.exp(-x))
    return x


def slope(kind, x):
    """d act / d x."""
    if kind == "exp":
        return np.exp(x)
    if kind == "sigmoid":
        s = 1.0 / (1.0 + np.exp(-x))
        return s * (1.0 - s)
    return np.ones_like(x)


def group_of(plane, row_index):
    """Group of row `row_index` (leading indices) of a plane."""
    if plane == "sh":
        return "SH_DC" if row_index[0] == 0 else "SH_REST"
    return {"mean": "MEAN", "scale": "SCALE", "rot": "ROT", "opacity": "OPACITY"}.get(plane, "SG")


def adam_step(raw, grad_act, m, v, lr, step, n, beta1=0.9, beta2=0.999, eps=1e-15):
    """One step over every plane present in `raw` (dicts of float64 arrays [..., stride]);
    entries [0, n) of each row are updated.  lr, step: dicts by group name.  Returns new
    (raw, act, m, v) dicts (the inputs are not modified)."""
    out_x, out_a, out_m, out_v = {}, {}, {}, {}
    for p, x in raw.items():
        if x is None:
            out_x[p] = out_a[p] = out_m[p] = out_v[p] = None
            continue
        kind = activation(p)
        x = np.array(x, np.float64)
        mm = np.array(m[p], np.float64)
        vv = np.array(v[p], np.float64)
        for idx in np.ndindex(x.shape[:-1]):
            grp = group_of(p, idx)
            if lr[grp] == 0.0:
                continue
            t = step[grp]
            xs = x[idx][:n]
            g = np.asarray(grad_act[p][idx][:n], np.float64) * slope(kind, xs)
            mrow = beta1 * mm[idx][:n] + (1.0 - beta1) * g
            vrow = beta2 * vv[idx][:n] + (1.0 - beta2) * g * g
            mhat = mrow / (1.0 - beta1 ** t)
            vhat = vrow / (1.0 - beta2 ** t)
            x[idx][:n] = xs - lr[grp] * mhat / (np.sqrt(vhat) + eps)
            mm[idx][:n] = mrow
            vv[idx][:n] = vrow
        out_x[p], out_a[p], out_m[p], out_v[p] = x, activate(kind, x), mm, vv
    return out_x, out_a, out_m, out_v
