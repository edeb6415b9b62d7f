"""DLSC relaxation (Sec. 3.3.2, Alg. 2) - placeholder until built."""


class DLSCLevel:
    def __init__(self, prob, l, params):
        raise NotImplementedError("DLSC oracle not built yet")
