"""GB300-native batched flexible-ligand docking (the dock-and-score step of EXSCALATE).

``lg``     ctypes binding of the C-ABI library liblgdock.so (include/lg.h).
``synth``  seeded synthetic pockets and ligand batches (inputs only).
"""
