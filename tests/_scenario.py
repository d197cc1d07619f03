"""Test helpers: run a workloads.Scenario on the oracle and compare results."""
import numpy as np

from oracle.oracle import OracleGrid


def oracle_from_scenario(sc, parity=True):
    return OracleGrid.from_scenario(sc, parity=parity)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
