"""Closed forms from the literature that the oracle pins use, written out
once here so that several pins share one copy.  Nothing here calls the
oracle."""

import numpy as np


def aharoni_dz(A, B, C):
    """Demagnetising factor along the C side of a uniformly magnetised
    rectangular prism with sides A, B, C: A. Aharoni, J. Appl. Phys. 83, 3432
    (1998), Eq. 1, in terms of the half-sides a, b, c.  A closed form derived
    independently of Newell's cell-pair functions f and g."""
    a, b, c = A / 2, B / 2, C / 2
    abc = np.sqrt(a * a + b * b + c * c)
    ab, bc, ac = np.sqrt(a * a + b * b), np.sqrt(b * b + c * c), np.sqrt(a * a + c * c)
    t = ((b * b - c * c) / (2 * b * c) * np.log((abc - a) / (abc + a))
         + (a * a - c * c) / (2 * a * c) * np.log((abc - b) / (abc + b))
         + b / (2 * c) * np.log((ab + a) / (ab - a))
         + a / (2 * c) * np.log((ab + b) / (ab - b))
         + c / (2 * a) * np.log((bc - b) / (bc + b))
         + c / (2 * b) * np.log((ac - a) / (ac + a))
         + 2 * np.arctan(a * b / (c * abc))
         + (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
         + (a * a + b * b - 2 * c * c) / (3 * a * b * c) * abc
         + c / (a * b) * (ac + bc)
         - (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c))
    return t / np.pi
