"""Grid descriptor shared by generators, oracle and CUDA path (plain data)."""
from dataclasses import dataclass


@dataclass(frozen=True)
class Grid:
    """Cartesian fine grid with a uniform primal coarse partition.

    dims      -- fine-grid extent per dimension (cells for cell-centred FV,
                 nodes for vertex-centred FE), x fastest.
    H         -- coarse block edge per dimension (cells, or elements for FE).
    centering -- 0 = cell-centred (FV), 1 = vertex-centred (FE nodes).
    ncomp     -- unknowns per fine point (1 = pressure, 3 = displacement).
    """
    dims: tuple
    H: tuple
    centering: int = 0
    ncomp: int = 1

    @property
    def dim(self):
        return len(self.dims)

    @property
    def n(self):
        r = 1
        for d in self.dims:
            r *= d
        return r

    @property
    def W(self):
        return 2 ** self.dim
