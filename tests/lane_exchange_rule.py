"""Which 4- and 5-target tensor-core blocks the planner gives lane-exchange
gathers: an independent statement of the rule the GPU and host tests check
the planner's records against."""


def lane_exchange_expected(n, qubits, ctrls):
    """(layout admits the lane exchange, the automatic rule picks it) for a
    block with these targets and controls: bit 0 must not be a control, the
    groups must fill tiles of 128, and after the element bit's exchange at
    most two lane bits may still hold targets; the automatic rule picks it
    for every 5-target block and for 4-target blocks with two or more
    targets among bits 1..3."""
    t = set(qubits)
    free = [q for q in range(64) if q not in t and q not in ctrls][:5]
    cube = sorted(t | set(free))
    fits = 0 not in ctrls and n - len(qubits) - len(ctrls) >= 7
    if fits:
        lanes = cube[1:6]
        if 0 not in t:
            lanes[[q in t for q in lanes].index(True)] = 0
        fits = sum(q in t for q in lanes) <= 2
    pays = len(qubits) == 5 or len(t & {1, 2, 3}) >= 2
    return fits, pays
