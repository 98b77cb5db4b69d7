"""GB300-native matrix-free CHNS (Cahn-Hilliard Navier-Stokes) operator apply and
Newton-Krylov Crank-Nicolson step on 2:1-balanced octrees."""
