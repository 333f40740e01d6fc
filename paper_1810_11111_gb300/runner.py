"""Set up a solve on the CUDA library from a workload description.

Marshalling only: builds the index set, the operators and the solver through
the C ABI, and loads the initial coefficients (projected on the device for
separable data, or copied from the seeded per-coefficient draws).
"""
import numpy as np
import torch

from . import sgkiif
from .workloads import coefficient_noise


class Problem:
    def __init__(self, cfg, precision=sgkiif.SGK_FP64, device=0, stream=None, bc=sgkiif.SGK_PERIODIC):
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self.cfg = cfg
        self.device = torch.device("cuda", device)
        self.ctx = sgkiif.Context(device, stream, precision)
        self.idx = sgkiif.IndexSet(self.ctx, cfg["d"], cfg["n"], cfg["k"])
        self.ops = [sgkiif.Operator(self.ctx, self.idx, kap, bc) for kap in cfg["kappas"]]
        self.solver = sgkiif.Solver(self.ctx, self.ops, cfg["reaction"], cfg["M"], cfg["dt"], cfg.get("opts"),
                                    cfg.get("scheme", sgkiif.SGK_IIF2), cfg.get("reaction_form", "quadrature"))
        self.nspecies = len(self.ops)
        self.dof = self.idx.dof
        self.U0 = self.initial_state()
        self.sources = self.source_terms()
        for s, (lam, S) in enumerate(self.sources):
            if len(lam):
                self.solver.set_source(s, lam, S.data_ptr())

    def initial_state(self):
        """Initial coefficients per species as FP64 device tensors."""
        out = []
        noise = None
        for s, init in enumerate(self.cfg["init"]):
            if "noise_seed" in init:
                if noise is None:
                    bases = [i["base"] for i in self.cfg["init"]]
                    noise = coefficient_noise(init["noise_seed"], self.dof, self.nspecies, bases)
                out.append(torch.from_numpy(noise[s]).to(self.device))
            else:
                t = torch.empty(self.dof, dtype=torch.float64, device=self.device)
                self.idx.project_separable(init["amp"], init["wavenum"], init["kind"], init.get("const", 0.0),
                                           t.data_ptr())
                out.append(t)
        return out

    def source_terms(self):
        """Per species (lambdas, S): the terms e^{lam t} g(x) of cfg["sources"]
        (dicts with lam and the separable g as in init), g projected on the
        device into the rows of S."""
        out = []
        for s in range(self.nspecies):
            terms = self.cfg.get("sources", [[]] * self.nspecies)[s]
            S = torch.empty((len(terms), self.dof), dtype=torch.float64, device=self.device)
            for m, g in enumerate(terms):
                self.idx.project_separable(g["amp"], g["wavenum"], g["kind"], g.get("const", 0.0), S[m].data_ptr())
            out.append(([float(g["lam"]) for g in terms], S))
        return out

    def reset(self):
        """The initial state at t = 0."""
        for s in range(self.nspecies):
            self.solver.set_state(s, dev_ptr=self.U0[s].data_ptr())
        self.solver.set_time(0.0)

    def state(self):
        return [self.solver.get_state(s) for s in range(self.nspecies)]

    def close(self):
        self.solver.close()
        for o in self.ops:
            o.close()
        self.idx.close()
        self.ctx.close()
