"""Loading helpers for the hand-derived fixtures under tests/golden."""
import json
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def frac_array(rows):
    return np.array([[float(Fraction(v)) for v in row] for row in rows])


def frac_vector(vals):
    return np.array([float(Fraction(v)) for v in vals])
