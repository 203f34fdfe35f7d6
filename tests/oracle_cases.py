"""Shared helpers for the oracle tests: workload dicts -> oracle objects."""
from oracle.cosmology import Cosmology
from paper_2511_10353_gb300.workloads import BBKS, EH_NW  # noqa: F401  (plain dicts)


def cosmology_from(c):
    """Oracle Cosmology from a workload's cosmology dict."""
    return Cosmology(c["omega_m"], c["h"], c["n_s"], c["sigma_8"], tf=c.get("tf", "bbks"),
                     omega_l=c.get("omega_l", -1.0), omega_b=c.get("omega_b", 0.049),
                     t_cmb=c.get("t_cmb", 2.7255))
