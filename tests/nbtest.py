"""Shared helpers of the test-suite: workload recipes (the configurations of
the benchmark, by size) and error metrics.  No model arithmetic lives here."""
import numpy as np

# name: (n_donor, n_accretor, q, f_donor, f_accretor, eps, dt, expand_rate,
#        expand_steps, sigma_v)
WORKLOADS = {
    # two spheres of 512 elements, q = 0.5, 100 steps (FP64 reference size)
    "binary_1k": (512, 512, 0.5, 0.8, 0.5, 0.01, 1e-3, 0.0, -1, 1e-3),
    # 65,536 elements, q = 0.3, donor 0.9 -> 1.15 r_L over 10,000 steps
    "binary_64k": (49152, 16384, 0.3, 0.9, 0.5, 0.005, 5e-4, 0.25 / 10000, 10000, 1e-3),
    # 1,048,576 elements, q = 0.2
    "binary_1m": (786432, 262144, 0.2, 0.95, 0.4, 0.005, 2.5e-4, 0.0, -1, 1e-3),
}


def workload_kwargs(name):
    nd, na, q, fd, fa, eps, dt, rate, cap, sig = WORKLOADS[name]
    desc = dict(n_donor=nd, n_accretor=na, q=q, f_donor=fd, f_accretor=fa,
                expand_rate=rate, expand_steps=cap, sigma_v=sig, seed=0, stream=0)
    params = dict(eps=eps, dt=dt, beta=0.5, G=1.0, kappa_gamma=8.0, rl_coeff=0.69)
    return desc, params


def rms_rel(a, ref):
    """sqrt(sum |a - ref|^2 / sum |ref|^2) over elements."""
    num = float(np.sum((np.asarray(a) - np.asarray(ref)) ** 2))
    den = float(np.sum(np.asarray(ref) ** 2))
    return np.sqrt(num / den) if den > 0 else np.sqrt(num)


def oracle_ic(orc, desc, params):
    return orc.make_ic(desc["n_donor"], desc["n_accretor"], desc["q"],
                       f_donor=desc["f_donor"], f_accretor=desc["f_accretor"],
                       sigma_v=desc["sigma_v"], seed=desc["seed"], stream=desc["stream"],
                       G=params["G"], kappa_gamma=params["kappa_gamma"],
                       rl_coeff=params["rl_coeff"], ecc=desc.get("ecc", 0.0),
                       no_spin=bool(params.get("flags", 0) & 2))
