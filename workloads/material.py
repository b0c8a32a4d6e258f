"""Material constants and load levels (project choices, in SI units).

The paper uses the Guccione law (Section 2) but prints no constants; it
defers to Guccione et al. 1991.  These values are this project's own choice,
of the order of the cardiac-mechanics benchmark literature, picked so that
the slab workloads converge in a few load steps at half of the paper's peak
activation.  They are inputs, shared by both implementations as data.
"""


def default_material():
    return {
        "C": 10.0e3,     # Pa, scale of the exponential term
        "bff": 8.0,      # fibre-fibre
        "bss": 2.0,      # sheet-sheet
        "bnn": 2.0,      # normal-normal
        "bfs": 4.0,      # fibre-sheet (weights E_fs^2 + E_sf^2)
        "bfn": 4.0,      # fibre-normal
        "bsn": 2.0,      # sheet-normal
        "B": 100.0e3,    # Pa, volumetric penalty in B/2 (J-1) log J
    }


# Peak activation of the paper's contraction test, gamma(t) = 6e4 min(t,.25)/.25
# (Section 5); the workloads run at half of it.
GAMMA_MAX = 6.0e4
