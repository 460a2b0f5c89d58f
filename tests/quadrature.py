"""Collapsed-coordinate Gauss-Legendre quadrature on the reference elements.

Independent of the oracle: used by the tests to integrate nodal bases exactly
(Duffy collapse of the tensor Gauss rule onto simplices)."""
import numpy as np


def rule(shape, n=8):
    x, w = np.polynomial.legendre.leggauss(n)
    if shape == "quad":
        X = np.array([(a, b) for b in x for a in x])
        W = np.array([wa * wb for wb in w for wa in w])
        return X, W
    if shape == "hex":
        X = np.array([(a, b, c) for c in x for b in x for a in x])
        W = np.array([wa * wb * wc for wc in w for wb in w for wa in w])
        return X, W
    if shape == "tri":
        X, W = [], []
        for b, wb in zip(x, w):
            for a, wa in zip(x, w):
                X.append(((1 + a) * (1 - b) / 2 - 1, b))
                W.append(wa * wb * (1 - b) / 2)
        return np.array(X), np.array(W)
    if shape == "tet":
        X, W = [], []
        for c, wc in zip(x, w):
            for b, wb in zip(x, w):
                for a, wa in zip(x, w):
                    y = (1 + b) * (1 - c) / 2 - 1
                    xx = (1 + a) * (-y - c) / 2 - 1
                    X.append((xx, y, c))
                    W.append(wa * wb * wc * (1 - c) / 2 * (-y - c) / 2)
        return np.array(X), np.array(W)
    if shape == "pri":
        Xt, Wt = rule("tri", n)
        X = np.array([(p[0], p[1], z) for z in x for p in Xt])
        W = np.array([wt * wz for wz in w for wt in Wt])
        return X, W
    raise ValueError(shape)
